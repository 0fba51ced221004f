/*
 * FP64 CPU oracle for the particle-resolved thermal lattice Boltzmann step of
 * Xu & Li, "Particle-resolved thermal lattice Boltzmann simulation using
 * OpenACC on multi-GPUs" (arXiv 2308.16597).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library of the package: it is a plain,
 * slow, obviously-correct restatement of the method, in the paper's order:
 *
 *   collide (Eq. f, Eq. g) -> stream -> curved bounce-back on particle links
 *   (Bouzidi quadratic, Sec. 2.3; Li thermal Dirichlet, Sec. 2.3) ->
 *   momentum-exchange force and torque (Eq. force, Eq. torque) ->
 *   rigid-particle update (Sec. 2.2, spring repulsion Sec. 2.4) ->
 *   refilling of newborn nodes (Sec. 2.5).
 *
 * Everything is double precision, compiled without FMA contraction.  Where
 * the paper leaves a detail open, the reading taken is stated at the function
 * that implements it.
 *
 * Lattice: D2Q9 e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1)
 * e6=(-1,1) e7=(-1,-1) e8=(1,-1); D2Q5 uses e0..e4.  Node (i,j) sits at (i,j),
 * i in [0,nx), j in [0,ny); y points up, gravity points down; cavity walls
 * sit half-way, at -1/2 and n-1/2.
 *
 * Parity status: every function below is pinned by a CPU test against a
 * closed form, an invariant, a textbook special case or brute force, except
 * the full coupled multi-step run with moving particles, which no closed form
 * fixes (parity unpinned beyond the component pins).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y; /* 1 = periodic in that axis, 0 = walls */
    double T_wall[4];               /* wall temperature at x-, x+, y-, y+ */
} orc_domain;

typedef struct {
    double x, y;       /* centre (lattice units) */
    double ux, uy;     /* translational velocity */
    double theta;      /* orientation angle */
    double omega;      /* angular velocity (z) */
    double r;          /* radius; for an ellipse the semi-major axis a */
    double rho;        /* density */
    double T;          /* surface temperature T_w */
    double b;          /* semi-minor axis of an ellipse (major axis along theta); 0 for a disk */
} orc_particle;

typedef struct {
    double nu;         /* kinematic viscosity */
    double alpha;      /* thermal diffusivity */
    double g;          /* gravitational acceleration */
    double beta;       /* thermal expansion coefficient */
    double T0;         /* reference temperature of the buoyancy term */
    double rho_f;      /* fluid density (particle gravity/buoyancy) */
    double T_init;     /* initial fluid temperature */
    double s_e, s_eps; /* MRT-f rates of the energy moments */
    double s_q;        /* MRT-f rate of the heat-flux moments; <= 0 selects 8(2-s_nu)/(8-s_nu) */
    double q_e, q_nu;  /* MRT-g rates of the two non-conserved higher moments */
    double eps_w;      /* repulsion stiffness */
    double s_rep;      /* repulsion threshold distance */
    double body_fx, body_fy; /* uniform body force density (tests) */
    int32_t fixed_particles; /* 1: particles are not moved (tests) */
    int32_t reserved;
} orc_params;

typedef struct orc_sim orc_sim;

/* --- whole simulation ---------------------------------------------------- */
orc_sim *orc_create(const orc_domain *d, const orc_particle *p, int32_t np,
                    const orc_params *prm);
void orc_destroy(orc_sim *s);
/* Advance nsteps time steps.  Returns 0, or a negative code when a particle
 * leaves the domain (-4) or a fixed-index line holds two links (-5). */
int orc_step(orc_sim *s, int32_t nsteps);
/* rho, ux, uy, T at every node, row-major [ny][nx]; NaN at solid nodes. */
void orc_get_fields(const orc_sim *s, double *rho, double *ux, double *uy, double *T);
void orc_get_particles(const orc_sim *s, orc_particle *out);
/* Hydrodynamic force (x,y) and torque of the last step, 3 doubles per particle. */
void orc_get_forces(const orc_sim *s, double *out);
void orc_get_owner(const orc_sim *s, int32_t *out);
/* Pre-collision distributions at the current time: f[9][ny][nx], g[5][ny][nx]. */
void orc_get_state(const orc_sim *s, double *f, double *g);
void orc_set_state(orc_sim *s, const double *f, const double *g);
/* Bounce-back fallback counters of the last step:
 * [0] Bouzidi quadratic->linear, [1] Bouzidi ->simple, [2] thermal ->halfway,
 * [3] refill quadratic->linear, [4] ->copy, [5] ->equilibrium, [6] newborn nodes,
 * [7] links. */
void orc_get_counters(const orc_sim *s, int64_t *out8);

/* --- geometry (pure functions of particle positions) ---------------------- */
/* owner[j*nx+i] = id of the particle whose disk holds node (i,j), else -1. */
void orc_raster(int32_t nx, int32_t ny, const orc_particle *p, int32_t np, int32_t *owner);
/* Size of the effective zone of a particle and its fixed slot capacity. */
int32_t orc_zone_size(double r);
int32_t orc_slot_capacity(double r);
/* Fixed index array of Sec. 3: per particle 12N-12 slots.  node = j*nx+i of
 * the fluid node, or -1; q = wall distance fraction rounded to float.
 * Returns the number of lines found holding more than one link (0 normally). */
int32_t orc_build_slots(int32_t nx, int32_t ny, const int32_t *owner,
                        const orc_particle *p, int32_t np,
                        int32_t *slot_node, float *slot_q);
/* Brute-force enumeration: every (fluid node, direction) whose neighbour is
 * owned by a particle.  Writes up to cap entries of (node, dir, particle) and
 * the double q; returns the total count. */
int64_t orc_links_bruteforce(int32_t nx, int32_t ny, const int32_t *owner,
                             const orc_particle *p, int32_t np, int64_t cap,
                             int32_t *node, int32_t *dir, int32_t *pid, double *q);
/* Wall distance fraction q along e_k from (i,j) to the circle (x,y,r). */
double orc_link_q(int32_t i, int32_t j, int32_t k, double x, double y, double r);
/* cos(theta), sin(theta) by Cody-Waite reduction to [-pi/4, pi/4] and Taylor
 * polynomials, in a fixed order of IEEE operations (the GPU repeats it
 * operation for operation, so both sides rotate ellipses identically). */
void orc_cos_sin(double theta, double *c, double *s);
/* Ellipse geometry (Sec. 2.6 elliptical particles): node inside the ellipse
 * of particle P; wall fraction q of the link (i, j) -> (i, j) + e_k; support
 * distance h(n) = max over the ellipse of (x - x_c) . n for a unit n. */
int32_t orc_in_particle(int32_t i, int32_t j, const orc_particle *P);
double orc_link_q_particle(int32_t i, int32_t j, int32_t k, const orc_particle *P);
double orc_support(const orc_particle *P, double nx, double ny);

/* --- node-level operators (exported for the pins) ------------------------- */
void orc_moment_matrices(double M[81], double Minv[81], double N[25], double Ninv[25]);
/* One MRT collision of f at a node with force density (Fx, Fy). */
void orc_collide_f(const double f[9], double Fx, double Fy, const orc_params *prm, double out[9]);
/* One MRT collision of g at a node with fluid velocity (ux, uy). */
void orc_collide_g(const double g[5], double ux, double uy, const orc_params *prm, double out[5]);
void orc_feq(double rho, double ux, double uy, double out[9]);
void orc_geq(double T, double ux, double uy, double out[5]);
/* Bouzidi quadratic bounce-back with fallbacks.  fk0 = f_k^+(x_f),
 * fk1 = f_k^+(x_f-e_k), fk2 = f_k^+(x_f-2e_k), fb0 = f_kbar^+(x_f),
 * fb1 = f_kbar^+(x_f-e_k); have1/have2 = availability of x_f-e_k / x_f-2e_k;
 * eu = e_kbar . u_w.  Returns f_kbar(x_f, t+1); *level = 0 quadratic,
 * 1 linear, 2 simple. */
double orc_bouzidi(double q, int32_t k, double fk0, double fk1, double fk2,
                   double fb0, double fb1, int32_t have1, int32_t have2,
                   double eu, int32_t *level);
/* Li et al. curved Dirichlet bounce-back for g, k in 1..4. */
double orc_thermal_bb(double q, double gk0, double gk1, double gb0, int32_t have1,
                      double Tw, int32_t *level);
/* Spring repulsion of Sec. 2.4 for gap |x_s|, threshold s, stiffness eps,
 * force scale C: returns the magnitude along the unit gap vector. */
double orc_repulsion(double gap, double s, double eps, double C);
/* Newton-Euler step of one disk under force (Fx, Fy) and torque Tz. */
void orc_integrate(const orc_particle *P, double Fx, double Fy, double Tz, orc_particle *R);
/* Refilling (Sec. 2.5): extrapolation direction e_c for offset (dx, dy) from
 * the particle centre, and the refilled f (fh before, f after the velocity
 * constraint) and g of one newborn node; see lbm_oracle.c. */
int32_t orc_refill_direction(double dx, double dy);
void orc_refill_node(const double y1[9], const double y2[9], const double y3[9], int32_t nvalid,
                     double uwx, double uwy, double Tw, double fh[9], double f[9], double g[5]);

#ifdef __cplusplus
}
#endif
#endif
