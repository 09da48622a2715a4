/*
 * maclab_oracle.c -- plain, slow, FP64 CPU oracle of one MacLABSWE step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  The CUDA library shares
 * no code, header or table with it.
 *
 * What it computes (Zhou, "Macroscopic lattice Boltzmann method for shallow
 * water equations (MacLABSWE)", arXiv:1902.02999):
 *
 *   h(x,t)      = sum_a f^eq_a(x - e_a dt, t - dt)
 *                 - (g/e^2) sum_a C_a hbar_a [z_b(x) - z_b(x - e_a dt)]
 *                 + (dt/e^2) sum_a C_a e_aj F_j                       (Eq. Mac.lb.6)
 *   h u_i(x,t)  = the same sum weighted by e_ai                        (Eq. Mac.lb.7)
 *
 * with f^eq from Eq. feq-full, C_a and lambda_a from Section 3, the force F
 * from Eqs. SWE-force, wind_u-stress and bed-stress, the centred force of
 * Eq. force-CS, hbar from Eq. h-bar, e = 6 nu / dx from Eq. mlb-viscosity and
 * dt = dx / e, and the boundary rules of Section 3 (bounce-back, physical
 * variables prescribed directly).  Readings taken where the paper is silent:
 *
 *   R1  D2Q9 numbering: c_0=(0,0), c_1=(1,0), c_2=(1,1), c_3=(0,1),
 *       c_4=(-1,1), c_5=(-1,0), c_6=(-1,-1), c_7=(0,-1), c_8=(1,-1); the
 *       opposite of a is a+4 (mod 8).  This is the numbering for which the
 *       south-wall unknowns of Section 3 are {2,3,4} and pair with {6,7,8}.
 *   R2  hbar and the centred force are taken at the old time level:
 *       hbar_a = (h(x) + h(x - c_a))/2, Fbar_a = (F(x) + F(x - c_a))/2, so
 *       one step is fully explicit.
 *   R3  Bounce-back (link-wise, tau = 1): when the source x - c_a is a solid
 *       node, or lies outside the grid behind a bounce-back edge, the missing
 *       f^eq_a(x - c_a) is replaced by f^eq_abar(x) of the node itself and
 *       that link carries no bed-slope and no force term.
 *   R4  Specular (free-slip) edge: the source outside the grid is the mirror
 *       image of the node inside (half-way wall), with the normal components
 *       of velocity and force reversed; every term of the link is kept.
 *       Periodic edge: the source wraps around.
 *   R5  No-slip node: h from the update, u = v = 0.
 *       Dirichlet node on a grid edge: the prescribed quantities take their
 *       value at the new time t_{n+1}; each unprescribed one takes the new
 *       value of the first node inward along the edge normal (zero normal
 *       gradient), in a second pass once the other nodes are updated.
 *       (Linear extrapolation from two inward nodes is unstable at a 2D
 *       depth boundary; the velocity of the node's own update with walled-off
 *       links misses the Section 4.1 level bound by two orders.)
 *
 * Every function below works in double precision and loops over nodes and
 * directions in the order the equations are written; there is no blocking,
 * no fusion and no reordering.  Compile with -O2 -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Section 3, D2Q9: lattice directions, C_a and lambda_a ------------- */
static const int CX[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
static const int CY[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};

static double coef_C(int a)      /* C_a = 1/3 for a odd, 1/12 for a even */
{
    return (a % 2 == 1) ? 1.0 / 3.0 : 1.0 / 12.0;
}
static double coef_lambda(int a) /* lambda_a = 1 for a odd, 1/4 for a even */
{
    return (a % 2 == 1) ? 1.0 : 0.25;
}
static int opposite(int a) { return a == 0 ? 0 : ((a + 3) % 8) + 1; }

/* direction whose lattice vector is (sx*c_x, sy*c_y) */
static int mirrored(int a, int sx, int sy)
{
    int b;
    for (b = 0; b < 9; ++b)
        if (CX[b] == sx * CX[a] && CY[b] == sy * CY[a]) return b;
    return -1;
}

/* node types and edge kinds (the oracle's own copy of the mask coding) */
enum { OT_SOLID = 0, OT_FLUID = 1, OT_NOSLIP = 2, OT_DIR_H = 3, OT_DIR_Q = 4, OT_DIR_HU = 5 };
enum { OE_BOUNCEBACK = 0, OE_SPECULAR = 1, OE_PERIODIC = 2 };
enum { OW = 0, OEAST = 1, OS = 2, ON = 3 };

typedef struct {
    int nx, ny;
    double dx;
    double e;          /* particle speed, Eq. mlb-viscosity: e = 6 nu / dx */
    double g;
    double rho_w, rho_a, Cw, wind_u, wind_v;  /* Eq. wind_u-stress */
    double Cb;         /* Eq. bed-stress, C_b = g / C_z^2 */
    double Omega;      /* Coriolis parameter, Eq. SWE-force */
    int edge[4];       /* W, E, S, N */
    /* Dirichlet data per edge: [edge][0=h,1=qx,2=qy][mean, amp, omega, phase] */
    double bc[4][3][4];
} oracle_problem;

/* ---- Eq. feq-full -------------------------------------------------------- */
void oracle_feq(double h, double u, double v, double e, double g, double out[9])
{
    int a;
    double uu = u * u + v * v;
    out[0] = h * (1.0 - 5.0 * g * h / (6.0 * e * e) - 2.0 * uu / (3.0 * e * e));
    for (a = 1; a < 9; ++a) {
        double ex = e * CX[a], ey = e * CY[a];
        double eu = ex * u + ey * v;
        out[a] = coef_lambda(a) * h *
                 (g * h / (6.0 * e * e) + eu / (3.0 * e * e) +
                  eu * eu / (2.0 * e * e * e * e) - uu / (6.0 * e * e));
    }
}

/* ---- Eqs. SWE-force, wind_u-stress, bed-stress --------------------------- */
void oracle_force(const oracle_problem* p, double h, double u, double v, double F[2])
{
    double wmag = sqrt(p->wind_u * p->wind_u + p->wind_v * p->wind_v);
    double twx = p->rho_a * p->Cw * p->wind_u * wmag;  /* tau_w,x */
    double twy = p->rho_a * p->Cw * p->wind_v * wmag;
    double umag = sqrt(u * u + v * v);
    double tbx = p->rho_w * p->Cb * u * umag;          /* tau_b,x */
    double tby = p->rho_w * p->Cb * v * umag;
    F[0] = twx / p->rho_w - tbx / p->rho_w + p->Omega * h * v;
    F[1] = twy / p->rho_w - tby / p->rho_w - p->Omega * h * u;
}

static double wave(const double w[4], double t)
{
    return w[0] + w[1] * sin(w[2] * t + w[3]);
}

/* Resolve the source node of link a at node (i,j): returns 1 and sets
 * (si,sj,sx,sy) when the link is usable (sx,sy = -1 where a specular edge
 * mirrors the source), 0 when the link bounces back (R3, R4). */
static int resolve_source(const oracle_problem* p, const uint8_t* type, int i, int j, int a,
                          int* si, int* sj, int* sx, int* sy)
{
    int ii = i - CX[a], jj = j - CY[a];
    *sx = 1;
    *sy = 1;
    if (ii < 0 || ii >= p->nx) {
        int ed = ii < 0 ? OW : OEAST;
        if (p->edge[ed] == OE_BOUNCEBACK) return 0;
        if (p->edge[ed] == OE_PERIODIC) {
            ii = (ii + p->nx) % p->nx;
        } else {                       /* specular: half-way mirror */
            ii = ii < 0 ? -1 - ii : 2 * p->nx - 1 - ii;
            *sx = -1;
        }
    }
    if (jj < 0 || jj >= p->ny) {
        int ed = jj < 0 ? OS : ON;
        if (p->edge[ed] == OE_BOUNCEBACK) return 0;
        if (p->edge[ed] == OE_PERIODIC) {
            jj = (jj + p->ny) % p->ny;
        } else {
            jj = jj < 0 ? -1 - jj : 2 * p->ny - 1 - jj;
            *sy = -1;
        }
    }
    if (type[(size_t)jj * p->nx + ii] == OT_SOLID) return 0;
    *si = ii;
    *sj = jj;
    return 1;
}

/* Edge of a Dirichlet node and its inward normal (W, E, S, N priority).
 * Returns -1 when the node is not on a grid edge. */
static int dirichlet_edge(const oracle_problem* p, int i, int j, int* di, int* dj)
{
    if (i == 0) { *di = 1; *dj = 0; return OW; }
    if (i == p->nx - 1) { *di = -1; *dj = 0; return OEAST; }
    if (j == 0) { *di = 0; *dj = 1; return OS; }
    if (j == p->ny - 1) { *di = 0; *dj = -1; return ON; }
    return -1;
}

/* One MacLABSWE step, state (h,u,v) at t_n -> (h1,u1,v1) at t_n + dt.
 * t_next is t_{n+1}, used for the prescribed Dirichlet values.
 * Returns 0, or -1 if a Dirichlet node is not on a grid edge or its
 * inward node is solid or Dirichlet. */
int oracle_step(const oracle_problem* p, const double* zb, const uint8_t* type,
                const double* h, const double* u, const double* v,
                double* h1, double* u1, double* v1, double t_next)
{
    const int nx = p->nx, ny = p->ny;
    const double e = p->e, g = p->g, dt = p->dx / p->e;
    int i, j, a;
    /* Every node reads only the old state and writes only its own new
     * value, so the rows are independent: the timing build (-fopenmp)
     * splits them over the host cores, with the same arithmetic per node;
     * the test build ignores the pragma. */
#pragma omp parallel for private(i, a) schedule(static)
    for (j = 0; j < ny; ++j) {
        for (i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            double fx[9], Fx[2], Sh, Shu, Shv;
            if (type[x] == OT_SOLID) {
                h1[x] = h[x];
                u1[x] = u[x];
                v1[x] = v[x];
                continue;
            }
            oracle_feq(h[x], u[x], v[x], e, g, fx);
            oracle_force(p, h[x], u[x], v[x], Fx);
            /* a = 0: e_0 = 0 and z_b(x) - z_b(x) = 0, so only f^eq_0 remains */
            Sh = fx[0];
            Shu = 0.0;
            Shv = 0.0;
            for (a = 1; a < 9; ++a) {
                double ex = e * CX[a], ey = e * CY[a];
                int si, sj, sx, sy;
                double fa;
                if (!resolve_source(p, type, i, j, a, &si, &sj, &sx, &sy)) {
                    fa = fx[opposite(a)];            /* R3 bounce-back */
                } else {
                    size_t s = (size_t)sj * nx + si;
                    double fs[9], Fs[2], hbar, bed, Fbar_x, Fbar_y, force;
                    oracle_feq(h[s], u[s], v[s], e, g, fs);
                    oracle_force(p, h[s], u[s], v[s], Fs);
                    /* f^eq_a at the (possibly mirrored) source */
                    fa = fs[mirrored(a, sx, sy)];
                    /* Eq. h-bar at the old level (R2) */
                    hbar = 0.5 * (h[x] + h[s]);
                    bed = -(g * hbar / (e * e)) * coef_C(a) * (zb[x] - zb[s]);
                    /* Eq. force-CS at the link midpoint (R2); mirrored source
                     * force has its normal component reversed (R4) */
                    Fbar_x = 0.5 * (Fx[0] + sx * Fs[0]);
                    Fbar_y = 0.5 * (Fx[1] + sy * Fs[1]);
                    force = (dt / (e * e)) * coef_C(a) * (ex * Fbar_x + ey * Fbar_y);
                    fa = fa + bed + force;
                }
                Sh += fa;        /* Eq. Mac.lb.6 */
                Shu += ex * fa;  /* Eq. Mac.lb.7 */
                Shv += ey * fa;
            }
            h1[x] = Sh;
            u1[x] = Shu / Sh;
            v1[x] = Shv / Sh;
            if (type[x] == OT_NOSLIP) {              /* R5 */
                u1[x] = 0.0;
                v1[x] = 0.0;
            }
        }
    }
    /* R5, second pass: Dirichlet nodes, once every other node holds its new
     * value.  The inward node must be non-solid and not Dirichlet. */
    for (j = 0; j < ny; ++j) {
        for (i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i, n1;
            int di, dj, ed;
            if (type[x] < OT_DIR_H || type[x] > OT_DIR_HU) continue;
            ed = dirichlet_edge(p, i, j, &di, &dj);
            if (ed < 0 || i + di < 0 || i + di >= nx || j + dj < 0 || j + dj >= ny) return -1;
            n1 = (size_t)(j + dj) * nx + (i + di);
            if (type[n1] == OT_SOLID || type[n1] >= OT_DIR_H) return -1;
            if (type[x] == OT_DIR_H) {
                h1[x] = wave(p->bc[ed][0], t_next);
                u1[x] = u1[n1];
                v1[x] = v1[n1];
            } else {
                double qx = wave(p->bc[ed][1], t_next), qy = wave(p->bc[ed][2], t_next);
                if (type[x] == OT_DIR_Q)
                    h1[x] = h1[n1];
                else
                    h1[x] = wave(p->bc[ed][0], t_next);
                u1[x] = qx / h1[x];
                v1[x] = qy / h1[x];
            }
        }
    }
    return 0;
}

/* Advance n steps in place from step index n0 (t_n = n * dt).
 * Returns 0, -1 (bad Dirichlet node) or -2 (out of memory). */
int oracle_run(const oracle_problem* p, const double* zb, const uint8_t* type,
               double* h, double* u, double* v, int64_t n0, int64_t n)
{
    size_t N = (size_t)p->nx * p->ny;
    double *h1 = malloc(N * sizeof(double)), *u1 = malloc(N * sizeof(double)),
           *v1 = malloc(N * sizeof(double));
    double dt = p->dx / p->e;
    int64_t k;
    int rc = 0;
    if (!h1 || !u1 || !v1) {
        free(h1); free(u1); free(v1);
        return -2;
    }
    for (k = 0; k < n && rc == 0; ++k) {
        rc = oracle_step(p, zb, type, h, u, v, h1, u1, v1, (double)(n0 + k + 1) * dt);
        memcpy(h, h1, N * sizeof(double));
        memcpy(u, u1, N * sizeof(double));
        memcpy(v, v1, N * sizeof(double));
    }
    free(h1); free(u1); free(v1);
    return rc;
}

/* Steady-state residual between two states and the mass of the second,
 * over non-solid nodes:
 *   out[0] = || (dh, d(hu), d(hv)) ||_2 / || (h1, h1 u1, h1 v1) ||_2
 *   out[1] = sum h1,   out[2] = max |u1|. */
void oracle_residual(const oracle_problem* p, const uint8_t* type,
                     const double* h0, const double* u0, const double* v0,
                     const double* h1, const double* u1, const double* v1, int interval, double out[3])
{
    size_t N = (size_t)p->nx * p->ny, x;
    double num = 0.0, den = 0.0, mass = 0.0, umax = 0.0;
    for (x = 0; x < N; ++x) {
        double dh, dqx, dqy, sp;
        if (type[x] == OT_SOLID) continue;
        dh = h1[x] - h0[x];
        dqx = h1[x] * u1[x] - h0[x] * u0[x];
        dqy = h1[x] * v1[x] - h0[x] * v0[x];
        num += dh * dh + dqx * dqx + dqy * dqy;
        den += h1[x] * h1[x] + (h1[x] * u1[x]) * (h1[x] * u1[x]) + (h1[x] * v1[x]) * (h1[x] * v1[x]);
        mass += h1[x];
        sp = sqrt(u1[x] * u1[x] + v1[x] * v1[x]);
        if (sp > umax) umax = sp;
    }
    /* R7: the change over an interval of `interval` steps (state 0 is the
     * state `interval` steps before state 1), per step */
    out[0] = den > 0.0 ? sqrt(num) / sqrt(den) / (double)interval : 0.0;
    out[1] = mass;
    out[2] = umax;
}

/*
 * Independent formulation for self-checking: the distribution form of
 * Eq. lb.1 with tau = 1 written as a PUSH (forward streaming) of nine
 * stored distributions, followed by the moments of Eqs. fea-0-h and
 * fea-0-v.  Restricted to all-fluid grids with periodic edges.
 * Each node x sends, in every direction a, f^eq_a(x) plus the bed and
 * force terms of its link to x + c_a; the receiving node sums.
 */
int oracle_step_push(const oracle_problem* p, const double* zb,
                     const double* h, const double* u, const double* v,
                     double* h1, double* u1, double* v1)
{
    const int nx = p->nx, ny = p->ny;
    const double e = p->e, g = p->g, dt = p->dx / p->e;
    size_t N = (size_t)nx * ny, x;
    double* f = calloc(9 * N, sizeof(double));
    int i, j, a;
    if (!f) return -2;
    for (j = 0; j < ny; ++j) {
        for (i = 0; i < nx; ++i) {
            double fe[9], Fx[2];
            x = (size_t)j * nx + i;
            oracle_feq(h[x], u[x], v[x], e, g, fe);
            oracle_force(p, h[x], u[x], v[x], Fx);
            for (a = 0; a < 9; ++a) {
                int ti = (i + CX[a] + nx) % nx, tj = (j + CY[a] + ny) % ny;
                size_t t = (size_t)tj * nx + ti;
                double Ft[2], val = fe[a];
                if (a != 0) {
                    oracle_force(p, h[t], u[t], v[t], Ft);
                    /* Eq. lb.1: -(g hbar / e^2) C_a [z_b(x + e_a dt) - z_b(x)] */
                    val += -(g * 0.5 * (h[t] + h[x]) / (e * e)) * coef_C(a) * (zb[t] - zb[x]);
                    val += (dt / (e * e)) * coef_C(a) *
                           (e * CX[a] * 0.5 * (Fx[0] + Ft[0]) + e * CY[a] * 0.5 * (Fx[1] + Ft[1]));
                }
                f[(size_t)a * N + t] = val;
            }
        }
    }
    for (x = 0; x < N; ++x) {
        double hs = 0.0, mx = 0.0, my = 0.0;
        for (a = 0; a < 9; ++a) {
            hs += f[(size_t)a * N + x];                /* Eq. fea-0-h */
            mx += e * CX[a] * f[(size_t)a * N + x];    /* Eq. fea-0-v */
            my += e * CY[a] * f[(size_t)a * N + x];
        }
        h1[x] = hs;
        u1[x] = mx / hs;
        v1[x] = my / hs;
    }
    free(f);
    return 0;
}

/*
 * eLABSWE with a general relaxation time tau (Eq. lb.1, Section 3), the
 * distribution form that MacLABSWE reduces when tau = 1 (Eq. Mac.lb.3).
 * Nine distributions per node, f[a * N + x].  One step, pulled at every
 * non-solid node x, direction a, source y = x - c_a:
 *
 *   f_a(x, t + dt) = f*_a(y) - (g hbar / e^2) C_a [z_b(x) - z_b(y)]
 *                    + (dt / e^2) C_a e_aj Fbar_j
 *   f*_a(y)        = f_a(y) - [f_a(y) - f^eq_a(y)] / tau     (collision at y)
 *
 * with hbar and Fbar at the old level (R2).  A source that is solid or
 * behind a bounce-back edge returns the node's own post-collision value of
 * the opposite direction, f*_abar(x), without bed or force term (R3 with
 * general tau); a specular source is the mirror image of the node inside,
 * so it supplies f*_{mirror(a)} there (R4); periodic sources wrap.  No-slip
 * and Dirichlet nodes are not part of this form: returns -3 if any exists.
 * Solid nodes keep their distributions.
 */
static void elab_moments_at(const double* f, size_t N, size_t x, double e, double* h, double* u, double* v)
{
    int a;
    double hs = 0.0, mx = 0.0, my = 0.0;
    for (a = 0; a < 9; ++a) {
        hs += f[(size_t)a * N + x];                  /* Eq. fea-0-h */
        mx += e * CX[a] * f[(size_t)a * N + x];      /* Eq. fea-0-v */
        my += e * CY[a] * f[(size_t)a * N + x];
    }
    *h = hs;
    *u = mx / hs;
    *v = my / hs;
}

static double elab_post(const oracle_problem* p, const double* f, size_t N, size_t x, int a, double tau)
{
    double h, u, v, fe[9];
    elab_moments_at(f, N, x, p->e, &h, &u, &v);
    oracle_feq(h, u, v, p->e, p->g, fe);
    return f[(size_t)a * N + x] - (f[(size_t)a * N + x] - fe[a]) / tau;
}

int oracle_elab_step(const oracle_problem* p, const double* zb, const uint8_t* type, double tau,
                     const double* f, double* f1)
{
    const int nx = p->nx, ny = p->ny;
    const double e = p->e, g = p->g, dt = p->dx / p->e;
    const size_t N = (size_t)nx * ny;
    int i, j, a;
    for (j = 0; j < ny; ++j)
        for (i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            if (type[x] != OT_SOLID && type[x] != OT_FLUID) return -3;
        }
    for (j = 0; j < ny; ++j) {
        for (i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            double hx, ux, vx, Fx[2];
            if (type[x] == OT_SOLID) {
                for (a = 0; a < 9; ++a) f1[(size_t)a * N + x] = f[(size_t)a * N + x];
                continue;
            }
            elab_moments_at(f, N, x, e, &hx, &ux, &vx);
            oracle_force(p, hx, ux, vx, Fx);
            f1[x] = elab_post(p, f, N, x, 0, tau);  /* a = 0: no streaming, no terms */
            for (a = 1; a < 9; ++a) {
                int si, sj, sx, sy;
                double val;
                if (!resolve_source(p, type, i, j, a, &si, &sj, &sx, &sy)) {
                    val = elab_post(p, f, N, x, opposite(a), tau);
                } else {
                    size_t s = (size_t)sj * nx + si;
                    double hs, us, vs, Fs[2], hbar, Fbx, Fby;
                    elab_moments_at(f, N, s, e, &hs, &us, &vs);
                    oracle_force(p, hs, us, vs, Fs);
                    val = elab_post(p, f, N, s, mirrored(a, sx, sy), tau);
                    hbar = 0.5 * (hx + hs);
                    val += -(g * hbar / (e * e)) * coef_C(a) * (zb[x] - zb[s]);
                    Fbx = 0.5 * (Fx[0] + sx * Fs[0]);
                    Fby = 0.5 * (Fx[1] + sy * Fs[1]);
                    val += (dt / (e * e)) * coef_C(a) * (e * CX[a] * Fbx + e * CY[a] * Fby);
                }
                f1[(size_t)a * N + x] = val;
            }
        }
    }
    return 0;
}

/* f = f^eq(h, u, v) at every node (the equilibrium start of a run) */
void oracle_elab_init(const oracle_problem* p, const double* h, const double* u, const double* v, double* f)
{
    size_t N = (size_t)p->nx * p->ny, x;
    int a;
    for (x = 0; x < N; ++x) {
        double fe[9];
        oracle_feq(h[x], u[x], v[x], p->e, p->g, fe);
        for (a = 0; a < 9; ++a) f[(size_t)a * N + x] = fe[a];
    }
}

/* h, u, v of every node from the distributions (Eqs. fea-0-h, fea-0-v) */
void oracle_elab_moments(const oracle_problem* p, const double* f, double* h, double* u, double* v)
{
    size_t N = (size_t)p->nx * p->ny, x;
    for (x = 0; x < N; ++x) elab_moments_at(f, N, x, p->e, &h[x], &u[x], &v[x]);
}

/*
 * Variant: hbar at the new time level, as Eq. h-bar writes it for the link
 * that carries f_a from y = x - c_a into x:
 *     hbar_a = (h(x, t + dt) + h(y, t)) / 2.
 * The bed term is the only place h(x, t + dt) enters, and it enters
 * linearly, so the new depth of each node solves one linear equation:
 *     h1 = A - (1/2) sum_a k_a h(y_a) - (1/2) h1 sum_a k_a,
 *     k_a = (g / e^2) C_a [z_b(x) - z_b(y_a)]   (usable links only),
 * A being every other term of Eq. Mac.lb.6; the momentum of Eq. Mac.lb.7
 * follows with the same hbar.  Everything else (links, forces, no-slip and
 * Dirichlet rules) is as in oracle_step.
 */
int oracle_step_newlevel(const oracle_problem* p, const double* zb, const uint8_t* type,
                         const double* h, const double* u, const double* v,
                         double* h1, double* u1, double* v1, double t_next)
{
    const int nx = p->nx, ny = p->ny;
    const double e = p->e, g = p->g, dt = p->dx / p->e;
    int i, j, a;
    for (j = 0; j < ny; ++j) {
        for (i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i;
            double fx[9], Fx[2], A, Ax, Ay, Pk, Px, Py, K, Kx, Ky, hn;
            if (type[x] == OT_SOLID) {
                h1[x] = h[x];
                u1[x] = u[x];
                v1[x] = v[x];
                continue;
            }
            oracle_feq(h[x], u[x], v[x], e, g, fx);
            oracle_force(p, h[x], u[x], v[x], Fx);
            A = fx[0];
            Ax = Ay = 0.0;
            Pk = Px = Py = 0.0;   /* -(1/2) sum k_a h(y_a), weighted by 1, e c_ax, e c_ay */
            K = Kx = Ky = 0.0;    /* sum k_a, weighted likewise */
            for (a = 1; a < 9; ++a) {
                double ex = e * CX[a], ey = e * CY[a];
                int si, sj, sx, sy;
                double fa, k;
                if (!resolve_source(p, type, i, j, a, &si, &sj, &sx, &sy)) {
                    fa = fx[opposite(a)];            /* R3 bounce-back */
                    A += fa;
                    Ax += ex * fa;
                    Ay += ey * fa;
                    continue;
                }
                {
                    size_t s = (size_t)sj * nx + si;
                    double fs[9], Fs[2], Fbar_x, Fbar_y;
                    oracle_feq(h[s], u[s], v[s], e, g, fs);
                    oracle_force(p, h[s], u[s], v[s], Fs);
                    Fbar_x = 0.5 * (Fx[0] + sx * Fs[0]);
                    Fbar_y = 0.5 * (Fx[1] + sy * Fs[1]);
                    fa = fs[mirrored(a, sx, sy)] +
                         (dt / (e * e)) * coef_C(a) * (ex * Fbar_x + ey * Fbar_y);
                    A += fa;
                    Ax += ex * fa;
                    Ay += ey * fa;
                    k = (g / (e * e)) * coef_C(a) * (zb[x] - zb[s]);
                    Pk += -0.5 * k * h[s];
                    Px += -0.5 * ex * k * h[s];
                    Py += -0.5 * ey * k * h[s];
                    K += k;
                    Kx += ex * k;
                    Ky += ey * k;
                }
            }
            hn = (A + Pk) / (1.0 + 0.5 * K);
            h1[x] = hn;
            u1[x] = (Ax + Px - 0.5 * hn * Kx) / hn;
            v1[x] = (Ay + Py - 0.5 * hn * Ky) / hn;
            if (type[x] == OT_NOSLIP) {              /* R5 */
                u1[x] = 0.0;
                v1[x] = 0.0;
            }
        }
    }
    /* R5 second pass, as in oracle_step */
    for (j = 0; j < ny; ++j) {
        for (i = 0; i < nx; ++i) {
            size_t x = (size_t)j * nx + i, n1;
            int di, dj, ed;
            if (type[x] < OT_DIR_H || type[x] > OT_DIR_HU) continue;
            ed = dirichlet_edge(p, i, j, &di, &dj);
            if (ed < 0 || i + di < 0 || i + di >= nx || j + dj < 0 || j + dj >= ny) return -1;
            n1 = (size_t)(j + dj) * nx + (i + di);
            if (type[n1] == OT_SOLID || type[n1] >= OT_DIR_H) return -1;
            if (type[x] == OT_DIR_H) {
                h1[x] = wave(p->bc[ed][0], t_next);
                u1[x] = u1[n1];
                v1[x] = v1[n1];
            } else {
                double qx = wave(p->bc[ed][1], t_next), qy = wave(p->bc[ed][2], t_next);
                if (type[x] == OT_DIR_Q)
                    h1[x] = h1[n1];
                else
                    h1[x] = wave(p->bc[ed][0], t_next);
                u1[x] = qx / h1[x];
                v1[x] = qy / h1[x];
            }
        }
    }
    return 0;
}
