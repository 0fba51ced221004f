/*
 * FP64 CPU oracle of the particle-resolved thermal LBM step (arXiv 2308.16597).
 * TEST INFRASTRUCTURE ONLY: see lbm_oracle.h.  Compiled with -ffp-contract=off
 * so that every geometric predicate and wall fraction is a sequence of
 * correctly rounded IEEE operations.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Lattices (Sec. 2.1: D2Q9 for the flow, D2Q5 for the temperature).        */
/* ------------------------------------------------------------------------- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* D2Q5 MRT (the paper defers N, Q and n_eq to its earlier work): the energy
 * moment of the equilibrium is a*T with a = -2, which fixes the weights
 * w0 = (1-a)/5 and w1..4 = (4+a)/20 and the lattice sound speed
 * c_sT^2 = (4+a)/10 of the diffusive scheme. */
static const double A5 = -2.0;
static double w5(int i) { return i == 0 ? (1.0 - A5) / 5.0 : (4.0 + A5) / 20.0; }
static double cs2T(void) { return (4.0 + A5) / 10.0; }
static const double CS2 = 1.0 / 3.0; /* D2Q9 c_s^2 */
static const double RHO0 = 1.0;      /* reference density of the wall term */

/* ------------------------------------------------------------------------- */
/* Moment matrices                                                           */
/* ------------------------------------------------------------------------- */
/* Gauss-Jordan inverse with partial pivoting of an n x n matrix. */
static void invert(int n, const double *a, double *inv)
{
    double w[9 * 18];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            w[r * 2 * n + c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(w[r * 2 * n + col]) > fabs(w[piv * 2 * n + col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = w[col * 2 * n + c];
                w[col * 2 * n + c] = w[piv * 2 * n + c];
                w[piv * 2 * n + c] = t;
            }
        double d = w[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) w[col * 2 * n + c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = w[r * 2 * n + col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) w[r * 2 * n + c] -= m * w[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = w[r * 2 * n + n + c];
}

/* D2Q9 moment basis (density, energy, energy square, x-momentum, x heat flux,
 * y-momentum, y heat flux, normal stress, shear stress), each row written as
 * the polynomial of the lattice velocity that defines it. */
static void build_M(double M[81])
{
    for (int i = 0; i < 9; ++i) {
        double ex = EX[i], ey = EY[i], e2 = ex * ex + ey * ey;
        M[0 * 9 + i] = 1.0;
        M[1 * 9 + i] = 3.0 * e2 - 4.0;
        M[2 * 9 + i] = (9.0 * e2 * e2 - 21.0 * e2 + 8.0) / 2.0;
        M[3 * 9 + i] = ex;
        M[4 * 9 + i] = (3.0 * e2 - 5.0) * ex;
        M[5 * 9 + i] = ey;
        M[6 * 9 + i] = (3.0 * e2 - 5.0) * ey;
        M[7 * 9 + i] = ex * ex - ey * ey;
        M[8 * 9 + i] = ex * ey;
    }
}

/* D2Q5 moment basis: temperature, two heat fluxes, energy, normal stress. */
static void build_N(double N[25])
{
    for (int i = 0; i < 5; ++i) {
        double ex = EX[i], ey = EY[i], e2 = ex * ex + ey * ey;
        N[0 * 5 + i] = 1.0;
        N[1 * 5 + i] = ex;
        N[2 * 5 + i] = ey;
        N[3 * 5 + i] = 5.0 * e2 - 4.0;
        N[4 * 5 + i] = ex * ex - ey * ey;
    }
}

typedef struct {
    double M[81], Minv[81], N[25], Ninv[25];
    double S[9], Q[5];
} orc_ops;

static void build_ops(const orc_params *prm, orc_ops *o)
{
    build_M(o->M);
    invert(9, o->M, o->Minv);
    build_N(o->N);
    invert(5, o->N, o->Ninv);
    double s_nu = 1.0 / (3.0 * prm->nu + 0.5);
    double s_e = prm->s_e > 0 ? prm->s_e : 1.0;
    double s_eps = prm->s_eps > 0 ? prm->s_eps : 1.0;
    double s_q = prm->s_q > 0 ? prm->s_q : 8.0 * (2.0 - s_nu) / (8.0 - s_nu);
    double S[9] = {0.0, s_e, s_eps, 0.0, s_q, 0.0, s_q, s_nu, s_nu};
    memcpy(o->S, S, sizeof S);
    double q_k = 1.0 / (prm->alpha / cs2T() + 0.5);
    double q_e = prm->q_e > 0 ? prm->q_e : 1.0;
    double q_nu = prm->q_nu > 0 ? prm->q_nu : 1.0;
    double Q[5] = {0.0, q_k, q_k, q_e, q_nu};
    memcpy(o->Q, Q, sizeof Q);
}

void orc_moment_matrices(double M[81], double Minv[81], double N[25], double Ninv[25])
{
    build_M(M);
    invert(9, M, Minv);
    build_N(N);
    invert(5, N, Ninv);
}

/* ------------------------------------------------------------------------- */
/* Equilibria and collisions (Eq. f, Eq. g)                                  */
/* ------------------------------------------------------------------------- */
void orc_feq(double rho, double ux, double uy, double out[9])
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        out[i] = W9[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

void orc_geq(double T, double ux, double uy, double out[5])
{
    for (int i = 0; i < 5; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        out[i] = w5(i) * T * (1.0 + eu / cs2T());
    }
}

/* Eq. f at one node: m = M f; rho = sum f; u = (sum e f + F/2)/rho (Sec. 2.1);
 * m+ = m - S (m - m_eq) + (I - S/2) F_m; f+ = M^-1 m+.  The paper defers M,
 * m_eq and the forcing to earlier work: M is the Lallemand-Luo D2Q9 basis,
 * m_eq the moments of the second-order equilibrium and F_m the moments of
 * the Guo forcing term. */
static void collide_f(const orc_ops *o, const double f[9], double Fx, double Fy, double out[9])
{
    double m[9];
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i) s += o->M[r * 9 + i] * f[i];
        m[r] = s;
    }
    double rho = m[0];
    double ux = (m[3] + 0.5 * Fx) / rho;
    double uy = (m[5] + 0.5 * Fy) / rho;
    double uu = ux * ux + uy * uy;
    double meq[9] = {rho,
                     -2.0 * rho + 3.0 * rho * uu,
                     rho - 3.0 * rho * uu,
                     rho * ux,
                     -rho * ux,
                     rho * uy,
                     -rho * uy,
                     rho * (ux * ux - uy * uy),
                     rho * ux * uy};
    double uF = ux * Fx + uy * Fy;
    double Fm[9] = {0.0,
                    6.0 * uF,
                    -6.0 * uF,
                    Fx,
                    -Fx,
                    Fy,
                    -Fy,
                    2.0 * (ux * Fx - uy * Fy),
                    ux * Fy + uy * Fx};
    double mp[9];
    for (int r = 0; r < 9; ++r)
        mp[r] = m[r] - o->S[r] * (m[r] - meq[r]) + (1.0 - 0.5 * o->S[r]) * Fm[r];
    for (int i = 0; i < 9; ++i) {
        double s = 0.0;
        for (int r = 0; r < 9; ++r) s += o->Minv[i * 9 + r] * mp[r];
        out[i] = s;
    }
}

/* Eq. g at one node: n = N g; n_eq = (T, T ux, T uy, a T, 0); n+ = n - Q (n - n_eq). */
static void collide_g(const orc_ops *o, const double g[5], double ux, double uy, double out[5])
{
    double n[5];
    for (int r = 0; r < 5; ++r) {
        double s = 0.0;
        for (int i = 0; i < 5; ++i) s += o->N[r * 5 + i] * g[i];
        n[r] = s;
    }
    double T = n[0];
    double neq[5] = {T, T * ux, T * uy, A5 * T, 0.0};
    double np_[5];
    for (int r = 0; r < 5; ++r) np_[r] = n[r] - o->Q[r] * (n[r] - neq[r]);
    for (int i = 0; i < 5; ++i) {
        double s = 0.0;
        for (int r = 0; r < 5; ++r) s += o->Ninv[i * 5 + r] * np_[r];
        out[i] = s;
    }
}

void orc_collide_f(const double f[9], double Fx, double Fy, const orc_params *prm, double out[9])
{
    orc_ops o;
    build_ops(prm, &o);
    collide_f(&o, f, Fx, Fy, out);
}

void orc_collide_g(const double g[5], double ux, double uy, const orc_params *prm, double out[5])
{
    orc_ops o;
    build_ops(prm, &o);
    collide_g(&o, g, ux, uy, out);
}

/* ------------------------------------------------------------------------- */
/* Curved-boundary rules (Sec. 2.3)                                          */
/* ------------------------------------------------------------------------- */
/* Bouzidi quadratic interpolated bounce-back.  When a stencil node is not a
 * fluid node the rule falls back to linear interpolation, then to simple
 * bounce-back, each with its own wall-velocity term. */
double orc_bouzidi(double q, int32_t k, double fk0, double fk1, double fk2, double fb0,
                   double fb1, int32_t have1, int32_t have2, double eu, int32_t *level)
{
    double wall = 2.0 * W9[k] * RHO0 * eu / CS2;
    if (q <= 0.5) {
        if (have1 && have2) {
            *level = 0;
            return q * (2.0 * q + 1.0) * fk0 + (1.0 - 4.0 * q * q) * fk1 -
                   q * (1.0 - 2.0 * q) * fk2 + wall;
        }
        if (have1) {
            *level = 1;
            return 2.0 * q * fk0 + (1.0 - 2.0 * q) * fk1 + wall;
        }
        *level = 2;
        return fk0 + wall;
    }
    if (have1) {
        *level = 0;
        double c = 1.0 / (q * (2.0 * q + 1.0));
        return c * fk0 + (2.0 * q - 1.0) / q * fb0 - (2.0 * q - 1.0) / (2.0 * q + 1.0) * fb1 +
               c * wall;
    }
    *level = 1;
    return fk0 / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * fb0 + wall / (2.0 * q);
}

/* Li et al. curved Dirichlet rule for g: c_d1 = -1, c_d2 = c_d3 = (2q-1)/(2q+1),
 * c_d4 = 2/(2q+1).  Without the node x_f - e_k it falls back to the half-way
 * anti-bounce-back, which is the same rule at q = 1/2. */
double orc_thermal_bb(double q, double gk0, double gk1, double gb0, int32_t have1, double Tw,
                      int32_t *level)
{
    double wT = 2.0 * w5(1) * Tw;
    if (have1) {
        *level = 0;
        double c23 = (2.0 * q - 1.0) / (2.0 * q + 1.0);
        double c4 = 2.0 / (2.0 * q + 1.0);
        return -gk0 + c23 * gk1 + c23 * gb0 + c4 * wT;
    }
    *level = 1;
    return -gk0 + wT;
}

/* Spring repulsion of Sec. 2.4: zero beyond the threshold, else
 * (C/eps) ((|x_s| - s)/s)^2 along the gap vector. */
double orc_repulsion(double gap, double s, double eps, double C)
{
    if (gap > s) return 0.0;
    double t = (gap - s) / s;
    return C / eps * t * t;
}

/* ------------------------------------------------------------------------- */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------- */
static int in_disk(int32_t i, int32_t j, double x, double y, double r)
{
    double dx = (double)i - x;
    double dy = (double)j - y;
    return dx * dx + dy * dy <= r * r;
}

/* An ellipse is a particle with 0 < b != r; everything else is a disk of
 * radius r. */
static int is_ellipse(const orc_particle *P) { return P->b > 0.0 && P->b != P->r; }

/* Cody-Waite argument reduction (pi/2 split into a 33-bit head and a tail, so
 * that k * head is exact for |k| < 2^20) and Taylor polynomials of sin and
 * cos on [-pi/4, pi/4] (terms to x^17 and x^16: truncation below 1e-17). */
void orc_cos_sin(double theta, double *c, double *s)
{
    const double two_over_pi = 0.63661977236758134308;
    const double pio2_hi = 1.5707963267341256e+00;
    const double pio2_lo = 6.0771005065061922e-11;
    double k = floor(theta * two_over_pi + 0.5);
    double t = (theta - k * pio2_hi) - k * pio2_lo;
    double t2 = t * t;
    /* sin t = t (1 - t2/3! (1 - t2/(4 5) (1 - ...))) written as Horner in t2 */
    double ps = 1.0 / 355687428096000.0;            /* 1/17! */
    ps = ps * t2 - 1.0 / 1307674368000.0;           /* 1/15! */
    ps = ps * t2 + 1.0 / 6227020800.0;              /* 1/13! */
    ps = ps * t2 - 1.0 / 39916800.0;                /* 1/11! */
    ps = ps * t2 + 1.0 / 362880.0;                  /* 1/9!  */
    ps = ps * t2 - 1.0 / 5040.0;                    /* 1/7!  */
    ps = ps * t2 + 1.0 / 120.0;                     /* 1/5!  */
    ps = ps * t2 - 1.0 / 6.0;                       /* 1/3!  */
    double sn = t + t * (t2 * ps);
    double pc = 1.0 / 20922789888000.0;             /* 1/16! */
    pc = pc * t2 - 1.0 / 87178291200.0;             /* 1/14! */
    pc = pc * t2 + 1.0 / 479001600.0;               /* 1/12! */
    pc = pc * t2 - 1.0 / 3628800.0;                 /* 1/10! */
    pc = pc * t2 + 1.0 / 40320.0;                   /* 1/8!  */
    pc = pc * t2 - 1.0 / 720.0;                     /* 1/6!  */
    pc = pc * t2 + 1.0 / 24.0;                      /* 1/4!  */
    pc = pc * t2 - 0.5;                             /* 1/2!  */
    double cn = 1.0 + t2 * pc;
    long long q = (long long)k & 3;
    if (q == 0) { *c = cn; *s = sn; }
    else if (q == 1) { *c = -sn; *s = cn; }
    else if (q == 2) { *c = -cn; *s = -sn; }
    else { *c = sn; *s = -cn; }
}

/* Offset of node (i, j) from the centre in the ellipse's frame (u along the
 * major axis). */
static void ellipse_frame(double dx, double dy, double c, double s, double *u, double *v)
{
    *u = dx * c + dy * s;
    *v = dy * c - dx * s;
}

/* Inside iff u^2 / a^2 + v^2 / b^2 <= 1, evaluated as u^2 b^2 + v^2 a^2 <=
 * a^2 b^2 (no division). */
static int in_ellipse(int32_t i, int32_t j, const orc_particle *P)
{
    double c, s, u, v;
    orc_cos_sin(P->theta, &c, &s);
    ellipse_frame((double)i - P->x, (double)j - P->y, c, s, &u, &v);
    double a2 = P->r * P->r, b2 = P->b * P->b;
    return u * u * b2 + v * v * a2 <= a2 * b2;
}

int32_t orc_in_particle(int32_t i, int32_t j, const orc_particle *P)
{
    return is_ellipse(P) ? in_ellipse(i, j, P) : in_disk(i, j, P->x, P->y, P->r);
}

/* Support distance of the particle along the unit vector (nx, ny): r for a
 * disk, sqrt(a^2 (n.u)^2 + b^2 (n.v)^2) for an ellipse. */
double orc_support(const orc_particle *P, double nx, double ny)
{
    if (!is_ellipse(P)) return P->r;
    double c, s, nu, nv;
    orc_cos_sin(P->theta, &c, &s);
    ellipse_frame(nx, ny, c, s, &nu, &nv);
    return sqrt(P->r * P->r * nu * nu + P->b * P->b * nv * nv);
}

void orc_raster(int32_t nx, int32_t ny, const orc_particle *p, int32_t np, int32_t *owner)
{
    for (int64_t n = 0; n < (int64_t)nx * ny; ++n) owner[n] = -1;
    for (int32_t k = 0; k < np; ++k) {
        int32_t i0 = (int32_t)floor(p[k].x - p[k].r) - 1, i1 = (int32_t)floor(p[k].x + p[k].r) + 1;
        int32_t j0 = (int32_t)floor(p[k].y - p[k].r) - 1, j1 = (int32_t)floor(p[k].y + p[k].r) + 1;
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > nx - 1) i1 = nx - 1;
        if (j1 > ny - 1) j1 = ny - 1;
        for (int32_t j = j0; j <= j1; ++j)
            for (int32_t i = i0; i <= i1; ++i)
                if (orc_in_particle(i, j, &p[k])) owner[(int64_t)j * nx + i] = k;
    }
}

/* Effective zone of Sec. 3: N = INT(x_c + r) - INT(x_c - r) + 3 for integer
 * radii; for any radius the bound ceil(2r) + 3 keeps the zone square and
 * holds every link source.  Capacity 4N + 4(2N - 3) = 12N - 12. */
int32_t orc_zone_size(double r) { return (int32_t)ceil(2.0 * r) + 3; }
int32_t orc_slot_capacity(double r) { return 12 * orc_zone_size(r) - 12; }

/* q = |x_f - x_w| / |x_f - x_b| (Sec. 2.3) for the disk (x, y, r): the
 * smaller root t of |d + t e|^2 = r^2, d = x_f - x_c, written in the form
 * t = (|d|^2 - r^2) / (-(d.e) + sqrt((d.e)^2 - |e|^2 (|d|^2 - r^2))),
 * which has no cancellation because d.e < 0 on every link. */
double orc_link_q(int32_t i, int32_t j, int32_t k, double x, double y, double r)
{
    double dx = (double)i - x;
    double dy = (double)j - y;
    double de = (double)EX[k] * dx + (double)EY[k] * dy;
    double a = (double)(EX[k] * EX[k] + EY[k] * EY[k]);
    double c = (dx * dx + dy * dy) - r * r;
    double disc = de * de - a * c;
    if (disc < 0.0) disc = 0.0;
    double t = c / (-de + sqrt(disc));
    if (t > 1.0) t = 1.0;
    return t;
}

/* q for a link to an ellipse: the smaller root t of F(d + t e) = 0 with
 * F(w) = u(w)^2 b^2 + v(w)^2 a^2 - a^2 b^2 (the ellipse frame), i.e.
 * P2 t^2 + 2 P1 t + P0 = 0, written t = P0 / (-P1 + sqrt(P1^2 - P2 P0));
 * P0 > 0 (x_f is outside) and P1 < 0 on a link, so there is no
 * cancellation.  For a disk the root is orc_link_q's. */
double orc_link_q_particle(int32_t i, int32_t j, int32_t k, const orc_particle *P)
{
    if (!is_ellipse(P)) return orc_link_q(i, j, k, P->x, P->y, P->r);
    double c, s, du, dv, eu, ev;
    orc_cos_sin(P->theta, &c, &s);
    ellipse_frame((double)i - P->x, (double)j - P->y, c, s, &du, &dv);
    ellipse_frame((double)EX[k], (double)EY[k], c, s, &eu, &ev);
    double a2 = P->r * P->r, b2 = P->b * P->b;
    double P2 = eu * eu * b2 + ev * ev * a2;
    double P1 = du * eu * b2 + dv * ev * a2;
    double P0 = du * du * b2 + dv * dv * a2 - a2 * b2;
    double disc = P1 * P1 - P2 * P0;
    if (disc < 0.0) disc = 0.0;
    double t = P0 / (-P1 + sqrt(disc));
    if (t > 1.0) t = 1.0;
    return t;
}

static int inside(int32_t nx, int32_t ny, int32_t i, int32_t j)
{
    return i >= 0 && i < nx && j >= 0 && j < ny;
}

/* Zone node (a, b) of the t-th point of line `line` for direction k:
 * e1/e3 run along rows (line = b), e2/e4 along columns (line = a),
 * e5/e7 along constant a - b (line = a - b + N - 2), e6/e8 along constant
 * a + b (line = a + b - 1).  The two one-node lines at the zone corners of
 * each diagonal family are left out, since a link there would have to reach
 * a node outside the disk's bounding box. */
static int zone_point(int32_t k, int32_t N, int32_t line, int32_t t, int32_t *a, int32_t *b)
{
    if (k == 1 || k == 3) {
        *a = t;
        *b = line;
    } else if (k == 2 || k == 4) {
        *a = line;
        *b = t;
    } else if (k == 5 || k == 7) {
        *a = t;
        *b = t - (line - (N - 2));
    } else {
        *a = t;
        *b = (line + 1) - t;
    }
    return *b >= 0 && *b < N;
}

int32_t orc_build_slots(int32_t nx, int32_t ny, const int32_t *owner, const orc_particle *p,
                        int32_t np, int32_t *slot_node, float *slot_q)
{
    int64_t base = 0;
    int32_t overflow = 0;
    for (int32_t pid = 0; pid < np; ++pid) {
        int32_t N = orc_zone_size(p[pid].r);
        int32_t X0 = (int32_t)floor(p[pid].x - p[pid].r) - 1;
        int32_t Y0 = (int32_t)floor(p[pid].y - p[pid].r) - 1;
        int64_t off = base;
        for (int32_t k = 1; k <= 8; ++k) {
            int32_t nlines = k <= 4 ? N : 2 * N - 3;
            for (int32_t line = 0; line < nlines; ++line) {
                int32_t found = 0, node = -1;
                float q = 0.0f;
                for (int32_t t = 0; t < N; ++t) {
                    int32_t a, b;
                    if (!zone_point(k, N, line, t, &a, &b)) continue;
                    int32_t i = X0 + a, j = Y0 + b;
                    if (!inside(nx, ny, i, j) || owner[(int64_t)j * nx + i] != -1) continue;
                    int32_t si = i + EX[k], sj = j + EY[k];
                    if (!inside(nx, ny, si, sj) || owner[(int64_t)sj * nx + si] != pid) continue;
                    if (++found == 1) {
                        node = j * nx + i;
                        q = (float)orc_link_q_particle(i, j, k, &p[pid]);
                    }
                }
                if (found > 1) ++overflow;
                slot_node[off + line] = node;
                slot_q[off + line] = q;
            }
            off += nlines;
        }
        base += orc_slot_capacity(p[pid].r);
    }
    return overflow;
}

int64_t orc_links_bruteforce(int32_t nx, int32_t ny, const int32_t *owner,
                             const orc_particle *p, int32_t np, int64_t cap, int32_t *node,
                             int32_t *dir, int32_t *pid, double *q)
{
    (void)np;
    int64_t n = 0;
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            if (owner[(int64_t)j * nx + i] != -1) continue;
            for (int32_t k = 1; k < 9; ++k) {
                int32_t si = i + EX[k], sj = j + EY[k];
                if (!inside(nx, ny, si, sj)) continue;
                int32_t o = owner[(int64_t)sj * nx + si];
                if (o < 0) continue;
                if (n < cap) {
                    node[n] = j * nx + i;
                    dir[n] = k;
                    pid[n] = o;
                    q[n] = orc_link_q_particle(i, j, k, &p[o]);
                }
                ++n;
            }
        }
    return n;
}

/* ------------------------------------------------------------------------- */
/* Simulation                                                                */
/* ------------------------------------------------------------------------- */
struct orc_sim {
    orc_domain d;
    orc_params prm;
    orc_ops ops;
    int32_t np;
    orc_particle *p;
    double *force; /* 3 per particle: Fx, Fy, Tz (hydrodynamic, last step) */
    int64_t nn;
    double *f, *g;         /* pre-collision, [9][nn], [5][nn] */
    double *fp, *gp;       /* post-collision */
    int32_t *owner, *owner_new;
    int64_t counters[8];
};

#define F(s, i, n) ((s)->f[(int64_t)(i) * (s)->nn + (n)])
#define G(s, i, n) ((s)->g[(int64_t)(i) * (s)->nn + (n)])
#define FP(s, i, n) ((s)->fp[(int64_t)(i) * (s)->nn + (n)])
#define GP(s, i, n) ((s)->gp[(int64_t)(i) * (s)->nn + (n)])

/* Buoyancy F = rho g beta (T - T0) y-hat (Sec. 2.1), y pointing up so that
 * hot fluid rises, plus the uniform body force of the tests. */
static void node_force(const orc_sim *s, double rho, double T, double *Fx, double *Fy)
{
    *Fx = s->prm.body_fx;
    *Fy = rho * s->prm.g * s->prm.beta * (T - s->prm.T0) + s->prm.body_fy;
}

orc_sim *orc_create(const orc_domain *d, const orc_particle *p, int32_t np, const orc_params *prm)
{
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->d = *d;
    s->prm = *prm;
    build_ops(prm, &s->ops);
    s->np = np;
    s->p = (orc_particle *)malloc(sizeof(orc_particle) * (np > 0 ? np : 1));
    if (np > 0) memcpy(s->p, p, sizeof(orc_particle) * np);
    s->force = (double *)calloc(3 * (size_t)(np > 0 ? np : 1), sizeof(double));
    s->nn = (int64_t)d->nx * d->ny;
    s->f = (double *)malloc(sizeof(double) * 9 * s->nn);
    s->g = (double *)malloc(sizeof(double) * 5 * s->nn);
    s->fp = (double *)malloc(sizeof(double) * 9 * s->nn);
    s->gp = (double *)malloc(sizeof(double) * 5 * s->nn);
    s->owner = (int32_t *)malloc(sizeof(int32_t) * s->nn);
    s->owner_new = (int32_t *)malloc(sizeof(int32_t) * s->nn);
    orc_raster(d->nx, d->ny, s->p, np, s->owner);
    double feq[9], geq[5];
    orc_feq(1.0, 0.0, 0.0, feq);
    orc_geq(prm->T_init, 0.0, 0.0, geq);
    for (int64_t n = 0; n < s->nn; ++n) {
        int solid = s->owner[n] >= 0;
        for (int i = 0; i < 9; ++i) F(s, i, n) = solid ? NAN : feq[i];
        for (int i = 0; i < 5; ++i) G(s, i, n) = solid ? NAN : geq[i];
    }
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->p);
    free(s->force);
    free(s->f);
    free(s->g);
    free(s->fp);
    free(s->gp);
    free(s->owner);
    free(s->owner_new);
    free(s);
}

/* Neighbour of node (i,j) at offset (dx,dy): its index, or -1 across a wall. */
static int64_t neighbour(const orc_sim *s, int32_t i, int32_t j, int32_t dx, int32_t dy)
{
    int32_t a = i + dx, b = j + dy;
    if (a < 0 || a >= s->d.nx) {
        if (!s->d.periodic_x) return -1;
        a = (a + s->d.nx) % s->d.nx;
    }
    if (b < 0 || b >= s->d.ny) {
        if (!s->d.periodic_y) return -1;
        b = (b + s->d.ny) % s->d.ny;
    }
    return (int64_t)b * s->d.nx + a;
}

/* Collision at every fluid node (Eq. f and Eq. g). */
static void collide_all(orc_sim *s)
{
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < s->nn; ++n) {
        if (s->owner[n] != -1) continue;
        double f[9], g[5], fo[9], go[5];
        double rho = 0.0, mx = 0.0, my = 0.0, T = 0.0;
        for (int i = 0; i < 9; ++i) {
            f[i] = F(s, i, n);
            rho += f[i];
            mx += EX[i] * f[i];
            my += EY[i] * f[i];
        }
        for (int i = 0; i < 5; ++i) {
            g[i] = G(s, i, n);
            T += g[i];
        }
        double Fx, Fy;
        node_force(s, rho, T, &Fx, &Fy);
        double ux = (mx + 0.5 * Fx) / rho, uy = (my + 0.5 * Fy) / rho;
        collide_f(&s->ops, f, Fx, Fy, fo);
        collide_g(&s->ops, g, ux, uy, go);
        for (int i = 0; i < 9; ++i) FP(s, i, n) = fo[i];
        for (int i = 0; i < 5; ++i) GP(s, i, n) = go[i];
    }
}

/* Streaming f_i(x + e_i, t+1) = f_i^+(x, t), written as a pull.  Links that
 * cross a cavity wall use half-way bounce-back for f (no-slip, wall at rest)
 * and half-way anti-bounce-back for g with the wall temperature.  Links from
 * a particle node are left as NaN: the particle rule of the next stage
 * overwrites every one of them. */
static void stream_all(orc_sim *s)
{
    const int32_t nx = s->d.nx, ny = s->d.ny;
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            int64_t n = (int64_t)j * nx + i;
            if (s->owner[n] != -1) continue;
            for (int k = 0; k < 9; ++k) {
                int64_t src = neighbour(s, i, j, -EX[k], -EY[k]);
                double v;
                if (src < 0) v = FP(s, OPP[k], n);
                else if (s->owner[src] != -1) v = NAN;
                else v = FP(s, k, src);
                F(s, k, n) = v;
            }
            for (int k = 0; k < 5; ++k) {
                int64_t src = neighbour(s, i, j, -EX[k], -EY[k]);
                double v;
                if (src < 0) {
                    /* the wall crossed by the pull from x - e_k */
                    int side = k == 1 ? 0 : k == 3 ? 1 : k == 2 ? 2 : 3;
                    v = -GP(s, OPP[k], n) + 2.0 * w5(k) * s->d.T_wall[side];
                } else if (s->owner[src] != -1) {
                    v = NAN;
                } else {
                    v = GP(s, k, src);
                }
                G(s, k, n) = v;
            }
        }
}

static int fluid_at(const orc_sim *s, const int32_t *own, int32_t i, int32_t j)
{
    return inside(s->d.nx, s->d.ny, i, j) && own[(int64_t)j * s->d.nx + i] == -1;
}

/* Curved bounce-back on every fluid-particle link found by brute force, and
 * the momentum-exchange force and torque of Eq. force / Eq. torque:
 *   dF = f_k^+(x_f,t)(e_k - u_w) - f_kbar(x_f,t+1)(e_kbar - u_w),
 *   dT = (x_w - x_c) x dF,
 * with x_w = x_f + q e_k and u_w = U + Omega x (x_w - x_c). */
static void particle_links(orc_sim *s)
{
    const int32_t nx = s->d.nx, ny = s->d.ny;
    for (int32_t p = 0; p < 3 * s->np; ++p) s->force[p] = 0.0;
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            int64_t n = (int64_t)j * nx + i;
            if (s->owner[n] != -1) continue;
            for (int32_t k = 1; k < 9; ++k) {
                int32_t si = i + EX[k], sj = j + EY[k];
                if (!inside(nx, ny, si, sj)) continue;
                int32_t pid = s->owner[(int64_t)sj * nx + si];
                if (pid < 0) continue;
                const orc_particle *P = &s->p[pid];
                int32_t kb = OPP[k];
                double q = orc_link_q_particle(i, j, k, P);
                double rx = ((double)i + q * EX[k]) - P->x;
                double ry = ((double)j + q * EY[k]) - P->y;
                double uwx = P->ux - P->omega * ry;
                double uwy = P->uy + P->omega * rx;
                int32_t i1 = i - EX[k], j1 = j - EY[k], i2 = i - 2 * EX[k], j2 = j - 2 * EY[k];
                int have1 = fluid_at(s, s->owner, i1, j1);
                int have2 = fluid_at(s, s->owner, i2, j2);
                int64_t n1 = have1 ? (int64_t)j1 * nx + i1 : n;
                int64_t n2 = have2 ? (int64_t)j2 * nx + i2 : n;
                double eu = -(EX[k] * uwx + EY[k] * uwy);
                int32_t lvl;
                double fk0 = FP(s, k, n);
                double fnew = orc_bouzidi(q, k, fk0, FP(s, k, n1), FP(s, k, n2), FP(s, kb, n),
                                          FP(s, kb, n1), have1, have2, eu, &lvl);
                if (lvl == 1) s->counters[0]++;
                if (lvl == 2) s->counters[1]++;
                F(s, kb, n) = fnew;
                if (k <= 4) {
                    int32_t tl;
                    G(s, kb, n) = orc_thermal_bb(q, GP(s, k, n), GP(s, k, n1), GP(s, kb, n), have1,
                                                 P->T, &tl);
                    if (tl) s->counters[2]++;
                }
                double dFx = fk0 * (EX[k] - uwx) - fnew * (EX[kb] - uwx);
                double dFy = fk0 * (EY[k] - uwy) - fnew * (EY[kb] - uwy);
                s->force[3 * pid + 0] += dFx;
                s->force[3 * pid + 1] += dFy;
                s->force[3 * pid + 2] += rx * dFy - ry * dFx;
                s->counters[7]++;
            }
        }
}

/* Newton-Euler update of one disk over one time step (Sec. 2.2, same time
 * step as the fluid).  The paper names no integrator; the reading taken:
 * U' = U + F/M, X' = X + (U + U')/2, Omega' = Omega + T/I,
 * theta' = theta + (Omega + Omega')/2, with M = rho_p pi r^2 and
 * I = M r^2 / 2 (a uniform disk); in 2-D the gyroscopic term vanishes. */
void orc_integrate(const orc_particle *P, double Fx, double Fy, double Tz, orc_particle *R)
{
    const double pi = 3.14159265358979323846;
    double M, I;
    if (is_ellipse(P)) { /* uniform ellipse: M = rho pi a b, I = M (a^2 + b^2) / 4 */
        M = P->rho * pi * P->r * P->b;
        I = 0.25 * M * (P->r * P->r + P->b * P->b);
    } else {
        M = P->rho * pi * P->r * P->r;
        I = 0.5 * M * P->r * P->r;
    }
    *R = *P;
    R->ux = P->ux + Fx / M;
    R->uy = P->uy + Fy / M;
    R->x = P->x + 0.5 * (P->ux + R->ux);
    R->y = P->y + 0.5 * (P->uy + R->uy);
    R->omega = P->omega + Tz / I;
    R->theta = P->theta + 0.5 * (P->omega + R->omega);
}

/* Rigid-particle update (Sec. 2.2) with the spring repulsion of Sec. 2.4.
 * Total force: hydrodynamic + buoyant weight -(rho_p - rho_f) pi r^2 g y-hat +
 * repulsion from the cavity walls and from other particles, then
 * orc_integrate. */
static int particle_update(orc_sim *s)
{
    const double pi = 3.14159265358979323846;
    const double sr = s->prm.s_rep, ew = s->prm.eps_w;
    const int32_t nx = s->d.nx, ny = s->d.ny;
    int bad = 0;
    orc_particle *np_ = (orc_particle *)malloc(sizeof(orc_particle) * (s->np > 0 ? s->np : 1));
    for (int32_t a = 0; a < s->np; ++a) {
        const orc_particle *P = &s->p[a];
        const double Aa = is_ellipse(P) ? pi * P->r * P->b : pi * P->r * P->r; /* area */
        double Ca = Aa * (P->rho - s->prm.rho_f) * s->prm.g;
        double Fx = s->force[3 * a + 0];
        double Fy = s->force[3 * a + 1] - (P->rho - s->prm.rho_f) * Aa * s->prm.g;
        double Tz = s->force[3 * a + 2];
        /* walls: the gap is the distance from the wall plane to the surface
         * (the support distance along the wall normal for an ellipse) */
        if (!s->d.periodic_x) {
            const double hx = orc_support(P, 1.0, 0.0);
            Fx += orc_repulsion((P->x + 0.5) - hx, sr, ew, Ca);
            Fx -= orc_repulsion(((double)nx - 0.5 - P->x) - hx, sr, ew, Ca);
        }
        if (!s->d.periodic_y) {
            const double hy = orc_support(P, 0.0, 1.0);
            Fy += orc_repulsion((P->y + 0.5) - hy, sr, ew, Ca);
            Fy -= orc_repulsion(((double)ny - 0.5 - P->y) - hy, sr, ew, Ca);
        }
        for (int32_t b = 0; b < s->np; ++b) {
            if (b == a) continue;
            const orc_particle *Q = &s->p[b];
            double dx = P->x - Q->x, dy = P->y - Q->y;
            double dist = sqrt(dx * dx + dy * dy);
            /* the gap along the line of centres: centre distance minus both
             * support distances along it (both radii for disks) */
            double gap = (is_ellipse(P) || is_ellipse(Q))
                             ? dist - orc_support(P, -dx / dist, -dy / dist) - orc_support(Q, dx / dist, dy / dist)
                             : dist - P->r - Q->r;
            if (gap > sr) continue;
            const double Ab = is_ellipse(Q) ? pi * Q->r * Q->b : pi * Q->r * Q->r;
            double Cb = Ab * (Q->rho - s->prm.rho_f) * s->prm.g;
            double mag = orc_repulsion(gap, sr, ew, 0.5 * (Ca + Cb));
            Fx += mag * dx / dist;
            Fy += mag * dy / dist;
        }
        orc_particle R = *P;
        if (!s->prm.fixed_particles) orc_integrate(P, Fx, Fy, Tz, &R);
        /* leaving the cavity: the zone (side from the major semi-axis) must
         * stay inside */
        if (R.x - R.r < -0.5 || R.x + R.r > (double)nx - 0.5 || R.y - R.r < -0.5 ||
            R.y + R.r > (double)ny - 0.5)
            bad = 1;
        np_[a] = R;
    }
    if (s->np > 0) memcpy(s->p, np_, sizeof(orc_particle) * s->np);
    free(np_);
    return bad;
}

/* Direction e_c of Sec. 2.5 for a newborn node at offset (dx, dy) from the
 * new particle centre: the largest n . e_c over the eight moving directions,
 * with n taken unnormalised (a positive scale does not change the argmax);
 * ties go to the lowest index. */
int32_t orc_refill_direction(double dx, double dy)
{
    int32_t c = 1;
    double best = (double)EX[1] * dx + (double)EY[1] * dy;
    for (int32_t k = 2; k < 9; ++k) {
        double v = (double)EX[k] * dx + (double)EY[k] * dy;
        if (v > best) {
            best = v;
            c = k;
        }
    }
    return c;
}

/* Refilled distributions of one newborn node (Sec. 2.5).  y1, y2, y3 hold
 * f at x + e_c, x + 2e_c, x + 3e_c at t+1; nvalid of them (from the first)
 * are fluid nodes at both times.  fh: the extrapolation (quadratic
 * 3 y1 - 3 y2 + y3; linear 2 y1 - y2; copy y1; or f_eq(1, u_w) when none is
 * usable).  f: fh with its two momentum moments replaced by rho u_w and all
 * other moments kept (the MRT velocity constraint).  g = g_eq(T_w, u_w). */
void orc_refill_node(const double y1[9], const double y2[9], const double y3[9], int32_t nvalid,
                     double uwx, double uwy, double Tw, double fh[9], double f[9], double g[5])
{
    double M[81], Minv[81], N[25], Ninv[25];
    orc_moment_matrices(M, Minv, N, Ninv);
    if (nvalid >= 3) {
        for (int k = 0; k < 9; ++k) fh[k] = 3.0 * y1[k] - 3.0 * y2[k] + y3[k];
    } else if (nvalid == 2) {
        for (int k = 0; k < 9; ++k) fh[k] = 2.0 * y1[k] - y2[k];
    } else if (nvalid == 1) {
        for (int k = 0; k < 9; ++k) fh[k] = y1[k];
    } else {
        orc_feq(1.0, uwx, uwy, fh);
    }
    double m[9];
    for (int r = 0; r < 9; ++r) {
        double a = 0.0;
        for (int k = 0; k < 9; ++k) a += M[r * 9 + k] * fh[k];
        m[r] = a;
    }
    m[3] = m[0] * uwx;
    m[5] = m[0] * uwy;
    for (int k = 0; k < 9; ++k) {
        double a = 0.0;
        for (int r = 0; r < 9; ++r) a += Minv[k * 9 + r] * m[r];
        f[k] = a;
    }
    orc_geq(Tw, uwx, uwy, g);
}

/* Refilling of newborn nodes (Sec. 2.5).  e_c maximises n . e_c over the
 * eight moving directions (n the outward normal, taken unnormalised; ties go
 * to the lowest index).  f is extrapolated quadratically from the nodes
 * x + e_c, x + 2e_c, x + 3e_c at t+1 (linear, then copy, then equilibrium at
 * the wall velocity when some of them are not fluid at both times); its two
 * momentum moments are then set to rho u_w, all other moments kept.
 * g = g_eq(T_w, u_w). */
static void refill(orc_sim *s)
{
    const int32_t nx = s->d.nx, ny = s->d.ny;
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            int64_t n = (int64_t)j * nx + i;
            int32_t pid = s->owner[n];
            if (pid < 0 || s->owner_new[n] != -1) continue;
            const orc_particle *P = &s->p[pid];
            s->counters[6]++;
            double dx = (double)i - P->x, dy = (double)j - P->y;
            /* outward normal: x - x_c for a disk; the gradient of the
             * ellipse function (u / a^2, v / b^2 in its frame) for an ellipse */
            int32_t c;
            if (is_ellipse(P)) {
                double cs, sn, u, v;
                orc_cos_sin(P->theta, &cs, &sn);
                ellipse_frame(dx, dy, cs, sn, &u, &v);
                double gu = u / (P->r * P->r), gv = v / (P->b * P->b);
                c = orc_refill_direction(gu * cs - gv * sn, gu * sn + gv * cs);
            } else {
                c = orc_refill_direction(dx, dy);
            }
            double uwx = P->ux - P->omega * dy;
            double uwy = P->uy + P->omega * dx;
            int64_t nb[3] = {n, n, n};
            int nvalid = 0;
            for (int m = 1; m <= 3; ++m) {
                int32_t a = i + m * EX[c], b = j + m * EY[c];
                if (!(fluid_at(s, s->owner, a, b) && fluid_at(s, s->owner_new, a, b))) break;
                nb[m - 1] = (int64_t)b * nx + a;
                nvalid = m;
            }
            if (nvalid == 2) s->counters[3]++;
            if (nvalid == 1) s->counters[4]++;
            if (nvalid == 0) s->counters[5]++;
            double y1[9], y2[9], y3[9], fh[9], fo[9], go[5];
            for (int k = 0; k < 9; ++k) {
                y1[k] = nvalid >= 1 ? F(s, k, nb[0]) : 0.0;
                y2[k] = nvalid >= 2 ? F(s, k, nb[1]) : 0.0;
                y3[k] = nvalid >= 3 ? F(s, k, nb[2]) : 0.0;
            }
            orc_refill_node(y1, y2, y3, nvalid, uwx, uwy, P->T, fh, fo, go);
            for (int k = 0; k < 9; ++k) F(s, k, n) = fo[k];
            for (int k = 0; k < 5; ++k) G(s, k, n) = go[k];
        }
}

int orc_step(orc_sim *s, int32_t nsteps)
{
    int rc = 0;
    for (int32_t t = 0; t < nsteps; ++t) {
        memset(s->counters, 0, sizeof s->counters);
        collide_all(s);
        stream_all(s);
        particle_links(s);
        if (particle_update(s)) rc = -4;
        orc_raster(s->d.nx, s->d.ny, s->p, s->np, s->owner_new);
        refill(s);
        /* covered nodes (fluid -> solid) are dropped */
        for (int64_t n = 0; n < s->nn; ++n)
            if (s->owner_new[n] != -1) {
                for (int i = 0; i < 9; ++i) F(s, i, n) = NAN;
                for (int i = 0; i < 5; ++i) G(s, i, n) = NAN;
            }
        int32_t *t_ = s->owner;
        s->owner = s->owner_new;
        s->owner_new = t_;
        if (rc) break;
    }
    return rc;
}

void orc_get_fields(const orc_sim *s, double *rho, double *ux, double *uy, double *T)
{
    for (int64_t n = 0; n < s->nn; ++n) {
        if (s->owner[n] != -1) {
            rho[n] = ux[n] = uy[n] = T[n] = NAN;
            continue;
        }
        double r = 0.0, mx = 0.0, my = 0.0, t = 0.0;
        for (int i = 0; i < 9; ++i) {
            r += F(s, i, n);
            mx += EX[i] * F(s, i, n);
            my += EY[i] * F(s, i, n);
        }
        for (int i = 0; i < 5; ++i) t += G(s, i, n);
        double Fx, Fy;
        node_force(s, r, t, &Fx, &Fy);
        rho[n] = r;
        ux[n] = (mx + 0.5 * Fx) / r;
        uy[n] = (my + 0.5 * Fy) / r;
        T[n] = t;
    }
}

void orc_get_particles(const orc_sim *s, orc_particle *out)
{
    if (s->np > 0) memcpy(out, s->p, sizeof(orc_particle) * s->np);
}

void orc_get_forces(const orc_sim *s, double *out)
{
    if (s->np > 0) memcpy(out, s->force, sizeof(double) * 3 * s->np);
}

void orc_get_owner(const orc_sim *s, int32_t *out)
{
    memcpy(out, s->owner, sizeof(int32_t) * s->nn);
}

void orc_get_state(const orc_sim *s, double *f, double *g)
{
    memcpy(f, s->f, sizeof(double) * 9 * s->nn);
    memcpy(g, s->g, sizeof(double) * 5 * s->nn);
}

void orc_set_state(orc_sim *s, const double *f, const double *g)
{
    memcpy(s->f, f, sizeof(double) * 9 * s->nn);
    memcpy(s->g, g, sizeof(double) * 5 * s->nn);
}

void orc_get_counters(const orc_sim *s, int64_t *out8)
{
    memcpy(out8, s->counters, sizeof s->counters);
}
