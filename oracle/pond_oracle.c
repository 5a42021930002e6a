/*
 * pond_oracle.c -- plain, slow FP64 reference implementation of the regularized
 * Particles-on-Demand finite-volume time step (Kallikounis, Dorschner, Karlin,
 * "Particles on Demand for flows with strong discontinuities", arXiv 2203.05477).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or helper with the CUDA library; every formula below is written out from
 * the paper, in population form, with no fusion or reordering beyond what the
 * paper states:
 *
 *   - lattice:      Table I (D1Q4 Gauss-Hermite roots and weights, T_L = 1) and
 *                   Eq. (wi) (D2Q16 as the tensor product W_i = w_ix w_iy; D3Q64, the
 *                   three-dimensional extension named as future work in Sec. V, as
 *                   W_i = w_ix w_iy w_iz);
 *   - velocities:   Eq. (vlambda)   v_i = sqrt(T/T_L) c_i + u;
 *   - moments:      Sec. II.B       rho, rho u, rho E;  Eq. (E) rho E = Cv rho T + rho u^2/2;
 *   - equilibria:   Eqs. (feqPond), (geqPond)   f^eq = rho W_i,  g^eq = (Cv - D/2) T rho W_i;
 *   - transform:    Eq. (f_transformed) with Eqs. (a0)-(a3): third-order Grad projection
 *                   for f, second-order for g (a3 dropped), built from the lab moments M_k;
 *   - FV update:    Eqs. (FinalUpdateDUGKS) in the co-moving frame (Sec. III.B.2);
 *   - flux:         Eqs. (InterfacePop), (FluxTransf), (Fbarplus), the face predictor-
 *                   corrector with limited slopes and MUSCL reconstruction (Sec. III.B.3),
 *                   and Eq. (fluxEq);
 *   - step order:   the algorithm summary of Sec. III.B.4;
 *   - time step:    CFL = max|v_ia| dt/dx (Sec. IV);
 *   - ablation:     the equilibration alternative of Sec. II.C (oracle_set_equilibration);
 *   - SL step:      the semi-Lagrangian realization of Sec. III.A (oracle_sl_step):
 *                   Eqs. (advectionPond)-(advectionPondg), (correctorfieldsrho)-
 *                   (correctorfieldT) and the BGK collision with beta.
 *
 * Readings where the paper is silent:
 *   R = 1, p = rho T, Cv = 1/(gamma-1); D in g^eq is the lattice dimension; the
 *   overline (symmetrization) is the sum over distinct index permutations; the face
 *   predictor before the first step is the frame of the pooled conserved moments of the two
 *   adjacent cells; a corrector pass whose moments define no frame (T <= 0 or not finite)
 *   restarts the corrector once from the frame of the pooled moments of the whole face
 *   stencil, and otherwise the corrector stops at the last pass that did define one; the
 *   corrector stops when |u_{k+1}-u_k|_inf <= tol sqrt(T_k) and |T_{k+1}-T_k| <= tol T_k,
 *   or after exactly `fixed_iters` passes when that is > 0; the face populations use the
 *   moments of the last pass, Grad-projected into the frame those moments define, with
 *   the co-moving equilibria there; van Leer (default) or minmod limiter on one-sided
 *   differences divided by the cell size; upwind cell = left/lower when v.n > 0, else
 *   right/upper; ghost cells (2 layers) are copies (transmissive), wraps (periodic),
 *   the equilibrium at a prescribed state (inflow), or mirror images (reflective walls:
 *   the normal component of every particle velocity and of the frame velocity reversed).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared pond_oracle.c -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define MAXQ 64
#define MAXD 3
#define NG 2

/* ------------------------------------------------------------------ lattice */

typedef struct {
    int D, Q;
    double TL;
    double c[MAXQ][MAXD];
    double W[MAXQ];
    int equilibrate;   /* 0: Grad's projection (the paper's choice); 1: the equilibration alternative */
} lattice;

/* Table I: D1Q4 nodes +-sqrt(3 -+ sqrt 6) with weights (3 +- sqrt 6)/12, T_L = 1.
 * D2Q16 (Eq. wi): population i = m*4 + n has c_i = (c_m, c_n), W_i = w_m w_n.
 * D3Q64 (the same product in three dimensions): i = (m*4 + n)*4 + p, c_i = (c_m, c_n, c_p),
 * W_i = w_m w_n w_p. */
static void lattice_init(lattice *L, int D)
{
    double s6 = sqrt(6.0);
    double c1[4] = {-sqrt(3.0 + s6), -sqrt(3.0 - s6), sqrt(3.0 - s6), sqrt(3.0 + s6)};
    double w1[4] = {(3.0 - s6) / 12.0, (3.0 + s6) / 12.0, (3.0 + s6) / 12.0, (3.0 - s6) / 12.0};
    memset(L, 0, sizeof(*L));
    L->D = D;
    L->TL = 1.0;
    if (D == 1) {
        L->Q = 4;
        for (int m = 0; m < 4; ++m) { L->c[m][0] = c1[m]; L->W[m] = w1[m]; }
    } else if (D == 2) {
        L->Q = 16;
        for (int m = 0; m < 4; ++m)
            for (int n = 0; n < 4; ++n) {
                int i = m * 4 + n;
                L->c[i][0] = c1[m];
                L->c[i][1] = c1[n];
                L->W[i] = w1[m] * w1[n];
            }
    } else {
        L->Q = 64;
        for (int m = 0; m < 4; ++m)
            for (int n = 0; n < 4; ++n)
                for (int p = 0; p < 4; ++p) {
                    int i = (m * 4 + n) * 4 + p;
                    L->c[i][0] = c1[m];
                    L->c[i][1] = c1[n];
                    L->c[i][2] = c1[p];
                    L->W[i] = w1[m] * w1[n] * w1[p];
                }
    }
}

static double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

/* ------------------------------------------------------- Grad transformation */

/* Sec. II.C: populations f_in known in frame lambda = (u_in, T_in) are re-expressed in
 * frame lambda' = (u_out, T_out) as the Grad projection Eq. (f_transformed) whose
 * coefficients are Eqs. (a0)-(a3) evaluated with the lab moments M_k of f_in.
 * order = 3 for f, 2 for g (the third-order term is dropped). */
static void grad_transform(const lattice *L, int order, const double *f_in,
                           const double *u_in, double T_in,
                           const double *u_out, double T_out, double *f_out)
{
    const int D = L->D, Q = L->Q;
    const double TL = L->TL;
    double M0 = 0.0, M1[MAXD] = {0}, M2[MAXD][MAXD] = {{0}}, M3[MAXD][MAXD][MAXD] = {{{0}}};
    const double sin_ = sqrt(T_in / TL);
    for (int i = 0; i < Q; ++i) {
        double v[MAXD];
        for (int a = 0; a < D; ++a) v[a] = sin_ * L->c[i][a] + u_in[a];
        M0 += f_in[i];
        for (int a = 0; a < D; ++a) {
            M1[a] += f_in[i] * v[a];
            for (int b = 0; b < D; ++b) {
                M2[a][b] += f_in[i] * v[a] * v[b];
                for (int c = 0; c < D; ++c) M3[a][b][c] += f_in[i] * v[a] * v[b] * v[c];
            }
        }
    }
    const double *up = u_out;
    const double r = sqrt(T_out / TL); /* (T'/T_L)^{1/2} */
    double a0, a1[MAXD], a2[MAXD][MAXD], a3[MAXD][MAXD][MAXD];
    /* Eq. (a0) */
    a0 = M0;
    /* Eq. (a1) */
    for (int a = 0; a < D; ++a) a1[a] = (M1[a] - M0 * up[a]) / r;
    /* Eq. (a2): overline(u' x a1) = u'_a a1_b + a1_a u'_b */
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b)
            a2[a][b] = (M2[a][b] - M0 * T_out * kd(a, b) - r * (up[a] * a1[b] + a1[a] * up[b])
                        - M0 * up[a] * up[b]) / (r * r);
    /* Eq. (a3): each overline is the sum over the three distinct index placements */
    memset(a3, 0, sizeof(a3));
    if (order >= 3) {
        double X[MAXD][MAXD];
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) X[a][b] = M0 * TL * kd(a, b) + a2[a][b];
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b)
                for (int c = 0; c < D; ++c) {
                    double t1 = up[a] * X[b][c] + up[b] * X[a][c] + up[c] * X[a][b];
                    double t2 = a1[a] * kd(b, c) + a1[b] * kd(a, c) + a1[c] * kd(a, b);
                    double t3 = a1[a] * up[b] * up[c] + up[a] * a1[b] * up[c] + up[a] * up[b] * a1[c];
                    a3[a][b][c] = (M3[a][b][c] - (r * r) * t1 - T_out * r * t2 - r * t3
                                   - M0 * up[a] * up[b] * up[c]) / (r * r * r);
                }
    }
    /* The equilibration alternative of Sec. II.C (an ablation; the paper uses Grad's
     * projection): the slow moments (orders <= order) are kept as above, and the fast ones
     * -- here the tensor Hermite components He_r(c_x) He_s(c_y) He_t(c_z) with r, s, t <= 3
     * and r + s + t > order, which the tensor-product lattices carry beyond the slow set --
     * take the values of the equilibrium with the same zeroth and first moments in the new
     * frame, M0 d_x^r d_y^s d_z^t with d = (M1/M0 - u') / sqrt(T'/T_L) (the Hermite
     * coefficients of a Maxwellian of temperature T' shifted by d).  D1Q4 carries no fast f
     * moment; its g has the order-3 one. */
    double fast[4][4][4];
    memset(fast, 0, sizeof(fast));
    if (L->equilibrate) {
        double d[MAXD] = {0};
        for (int a = 0; a < D; ++a) d[a] = (M1[a] / M0 - up[a]) / r;
        for (int rr = 0; rr <= 3; ++rr)
            for (int ss = 0; ss <= (D >= 2 ? 3 : 0); ++ss)
                for (int tt = 0; tt <= (D == 3 ? 3 : 0); ++tt)
                    if (rr + ss + tt > order)
                        fast[rr][ss][tt] = M0 * pow(d[0], rr) * (D >= 2 ? pow(d[1], ss) : 1.0) * (D == 3 ? pow(d[2], tt) : 1.0);
    }
    /* Eq. (f_transformed) */
    for (int i = 0; i < Q; ++i) {
        const double *c = L->c[i];
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int a = 0; a < D; ++a) {
            s1 += a1[a] * c[a];
            for (int b = 0; b < D; ++b) {
                s2 += a2[a][b] * (c[a] * c[b] - TL * kd(a, b));
                if (order >= 3)
                    for (int cc = 0; cc < D; ++cc)
                        s3 += a3[a][b][cc] * (c[a] * c[b] * c[cc]
                                              - TL * (c[a] * kd(b, cc) + c[b] * kd(a, cc) + c[cc] * kd(a, b)));
            }
        }
        double sf = 0.0;
        if (L->equilibrate) {
            /* probabilists' Hermite polynomials He_0..He_3 over k! at the node (T_L = 1) */
            const double hx[4] = {1.0, c[0], (c[0] * c[0] - 1.0) / 2.0, (c[0] * c[0] * c[0] - 3.0 * c[0]) / 6.0};
            double hy[4] = {1.0, 0.0, 0.0, 0.0}, hz[4] = {1.0, 0.0, 0.0, 0.0};
            if (D >= 2) {
                hy[1] = c[1]; hy[2] = (c[1] * c[1] - 1.0) / 2.0; hy[3] = (c[1] * c[1] * c[1] - 3.0 * c[1]) / 6.0;
            }
            if (D == 3) {
                hz[1] = c[2]; hz[2] = (c[2] * c[2] - 1.0) / 2.0; hz[3] = (c[2] * c[2] * c[2] - 3.0 * c[2]) / 6.0;
            }
            for (int rr = 0; rr <= 3; ++rr)
                for (int ss = 0; ss <= 3; ++ss)
                    for (int tt = 0; tt <= 3; ++tt) sf += fast[rr][ss][tt] * hx[rr] * hy[ss] * hz[tt];
        }
        f_out[i] = L->W[i] * (a0 + s1 / TL + s2 / (2.0 * TL * TL) + s3 / (6.0 * TL * TL * TL) + sf);
    }
}

/* Sec. II.B: rho, rho u, rho E of (f, g) given in frame (u, T). */
static void conserved_moments(const lattice *L, const double *f, const double *g,
                              const double *u, double T, double *rho, double *mom, double *rhoE)
{
    const int D = L->D, Q = L->Q;
    double s = sqrt(T / L->TL);
    double r = 0.0, m[MAXD] = {0}, e = 0.0;
    for (int i = 0; i < Q; ++i) {
        double v2 = 0.0;
        for (int a = 0; a < D; ++a) {
            double v = s * L->c[i][a] + u[a];
            m[a] += f[i] * v;
            v2 += v * v;
        }
        r += f[i];
        e += 0.5 * v2 * f[i] + g[i];
    }
    *rho = r;
    for (int a = 0; a < D; ++a) mom[a] = m[a];
    *rhoE = e;
}

/* Eq. (E) solved for T with R = 1, Cv = 1/(gamma-1). */
static double temperature_from(double rho, const double *mom, double rhoE, int D, double Cv)
{
    double k = 0.0;
    for (int a = 0; a < D; ++a) k += mom[a] * mom[a];
    return (rhoE - 0.5 * k / rho) / (Cv * rho);
}

/* Eqs. (feqPond), (geqPond) in the co-moving frame. */
static void equilibria(const lattice *L, double rho, double T, double Cv, double *feq, double *geq)
{
    for (int i = 0; i < L->Q; ++i) {
        feq[i] = rho * L->W[i];
        geq[i] = (Cv - 0.5 * L->D) * T * rho * L->W[i];
    }
}

/* Slope limiters named in Sec. III.B.3 (van Leer; minmod). a, b: one-sided slopes. */
static double limiter(int kind, double a, double b)
{
    if (kind == 1) { /* minmod */
        if (a * b <= 0.0) return 0.0;
        return fabs(a) < fabs(b) ? a : b;
    }
    /* van Leer: (sgn a + sgn b) |a||b| / (|a| + |b|) */
    double den = fabs(a) + fabs(b);
    if (den == 0.0) return 0.0;
    double sa = (a > 0.0) - (a < 0.0), sb = (b > 0.0) - (b < 0.0);
    return (sa + sb) * fabs(a) * fabs(b) / den;
}

/* --------------------------------------------------------------- the solver */

enum { BC_TRANSMISSIVE = 0, BC_PERIODIC = 1, BC_INFLOW = 2, BC_REFLECTIVE = 3 };

typedef struct oracle {
    lattice L;
    int D, Q, nx, ny, nz;
    int gx, gy, gz;    /* ghost layers in x, y and z (0 along the axes a grid does not have) */
    int px, py, pz;    /* padded extents */
    double dx, dy, dz, gamma, Cv, tau, cfl, t_end;
    int bc[6];         /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi */
    double inflow[4][4];
    int inflow_lo[4], inflow_hi[4];
    int limiter;
    double tol;
    int max_iter, fixed_iters;
    /* cell state (padded, AoS): populations in the cell frame (u, T) */
    double *f, *g, *u, *T;
    double *fp, *gp;   /* phi-bar-plus, Eq. (Fbarplus); the new populations in the SL step */
    double *un, *Tn;   /* the new frames in the SL step */
    /* faces: x-faces (nx+1) x ny x nz, y-faces nx x (ny+1) x nz, z-faces nx x ny x (nz+1);
     * gauge and populations */
    double *xu, *xT, *yu, *yT, *zu, *zT;
    double *xf, *xg, *yf, *yg, *zf, *zg;
    double t, dt, last_dt, forced_dt;
    long long steps, face_iters, face_count, nonconv, nonphys, fallbacks;
} oracle;

static int cidx3(const oracle *o, int i, int j, int k)
{
    return ((k + o->gz) * o->py + (j + o->gy)) * o->px + (i + o->gx);
}
static int cidx(const oracle *o, int i, int j) { return cidx3(o, i, j, 0); }
static int xface3(const oracle *o, int i, int j, int k) { return (k * o->ny + j) * (o->nx + 1) + i; }
static int yface3(const oracle *o, int i, int j, int k) { return (k * (o->ny + 1) + j) * o->nx + i; }
static int zface3(const oracle *o, int i, int j, int k) { return (k * o->ny + j) * o->nx + i; }
static int xface(const oracle *o, int i, int j) { return xface3(o, i, j, 0); }
static int yface(const oracle *o, int i, int j) { return yface3(o, i, j, 0); }

static void set_equilibrium_cell(oracle *o, int c, double rho, const double *u, double p)
{
    double T = p / rho;
    equilibria(&o->L, rho, T, o->Cv, o->f + (size_t)c * o->Q, o->g + (size_t)c * o->Q);
    for (int a = 0; a < o->D; ++a) o->u[(size_t)c * MAXD + a] = u[a];
    o->T[c] = T;
}

static void copy_cell(oracle *o, int dst, int src)
{
    memcpy(o->f + (size_t)dst * o->Q, o->f + (size_t)src * o->Q, sizeof(double) * o->Q);
    memcpy(o->g + (size_t)dst * o->Q, o->g + (size_t)src * o->Q, sizeof(double) * o->Q);
    memcpy(o->u + (size_t)dst * MAXD, o->u + (size_t)src * MAXD, sizeof(double) * MAXD);
    o->T[dst] = o->T[src];
}

/* Specular reflection at a wall normal to axis: the ghost holds the mirror image of the
 * source cell, population v_i taking the value of the population with the normal
 * component of c reversed, and the frame velocity's normal component reversed (reading
 * of reflective walls, Sec. IV, two-blast-wave and explosion-in-a-box cases). */
static void mirror_cell(oracle *o, int dst, int src, int axis)
{
    const lattice *L = &o->L;
    double f[MAXQ], g[MAXQ];
    for (int i = 0; i < o->Q; ++i) {
        int j = -1;
        for (int k = 0; k < o->Q; ++k) {
            int same = L->c[k][axis] == -L->c[i][axis];
            for (int a = 0; a < o->D; ++a)
                if (a != axis && L->c[k][a] != L->c[i][a]) same = 0;
            if (same) j = k;
        }
        f[i] = o->f[(size_t)src * o->Q + j];
        g[i] = o->g[(size_t)src * o->Q + j];
    }
    memcpy(o->f + (size_t)dst * o->Q, f, sizeof(double) * o->Q);
    memcpy(o->g + (size_t)dst * o->Q, g, sizeof(double) * o->Q);
    memcpy(o->u + (size_t)dst * MAXD, o->u + (size_t)src * MAXD, sizeof(double) * MAXD);
    o->u[(size_t)dst * MAXD + axis] = -o->u[(size_t)src * MAXD + axis];
    o->T[dst] = o->T[src];
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int wrapi(int v, int n) { return ((v % n) + n) % n; }

/* Two ghost layers: x-sides first (interior rows), then y-sides for every padded column,
 * then (3D) z-sides for every padded x-y position. */
static void fill_ghosts(oracle *o)
{
    for (int kz = 0; kz < o->nz; ++kz)
        for (int j = 0; j < o->ny; ++j)
            for (int k = 1; k <= o->gx; ++k) {
                for (int side = 0; side < 2; ++side) {
                    int i = side == 0 ? -k : o->nx - 1 + k;
                    int dst = cidx3(o, i, j, kz);
                    int b = o->bc[side];
                    if (b == BC_INFLOW && j >= o->inflow_lo[side] && j < o->inflow_hi[side]) {
                        double uu[3] = {o->inflow[side][1], o->inflow[side][2], 0.0};
                        set_equilibrium_cell(o, dst, o->inflow[side][0], uu, o->inflow[side][3]);
                    } else if (b == BC_PERIODIC) {
                        copy_cell(o, dst, cidx3(o, wrapi(i, o->nx), j, kz));
                    } else if (b == BC_REFLECTIVE) {
                        /* ghost -k mirrors cell k-1; ghost nx-1+k mirrors cell nx-k (clamped
                         * into the grid when it is thinner than the ghost layers) */
                        mirror_cell(o, dst, cidx3(o, clampi(side == 0 ? k - 1 : o->nx - k, 0, o->nx - 1), j, kz), 0);
                    } else {
                        copy_cell(o, dst, cidx3(o, clampi(i, 0, o->nx - 1), j, kz));
                    }
                }
            }
    if (o->D < 2) return;
    for (int kz = 0; kz < o->nz; ++kz)
        for (int i = -o->gx; i < o->nx + o->gx; ++i)
            for (int k = 1; k <= o->gy; ++k) {
                for (int side = 2; side < 4; ++side) {
                    int j = side == 2 ? -k : o->ny - 1 + k;
                    int dst = cidx3(o, i, j, kz);
                    int b = o->bc[side];
                    int ic = clampi(i, 0, o->nx - 1);
                    if (b == BC_INFLOW && ic >= o->inflow_lo[side] && ic < o->inflow_hi[side]) {
                        double uu[3] = {o->inflow[side][1], o->inflow[side][2], 0.0};
                        set_equilibrium_cell(o, dst, o->inflow[side][0], uu, o->inflow[side][3]);
                    } else if (b == BC_PERIODIC) {
                        copy_cell(o, dst, cidx3(o, i, wrapi(j, o->ny), kz));
                    } else if (b == BC_REFLECTIVE) {
                        mirror_cell(o, dst, cidx3(o, i, clampi(side == 2 ? k - 1 : o->ny - k, 0, o->ny - 1), kz), 1);
                    } else {
                        copy_cell(o, dst, cidx3(o, i, clampi(j, 0, o->ny - 1), kz));
                    }
                }
            }
    if (o->D < 3) return;
    for (int j = -o->gy; j < o->ny + o->gy; ++j)
        for (int i = -o->gx; i < o->nx + o->gx; ++i)
            for (int k = 1; k <= o->gz; ++k) {
                for (int side = 4; side < 6; ++side) {
                    int kz = side == 4 ? -k : o->nz - 1 + k;
                    int dst = cidx3(o, i, j, kz);
                    int b = o->bc[side];
                    if (b == BC_PERIODIC) {
                        copy_cell(o, dst, cidx3(o, i, j, wrapi(kz, o->nz)));
                    } else if (b == BC_REFLECTIVE) {
                        mirror_cell(o, dst, cidx3(o, i, j, clampi(side == 4 ? k - 1 : o->nz - k, 0, o->nz - 1)), 2);
                    } else {
                        copy_cell(o, dst, cidx3(o, i, j, clampi(kz, 0, o->nz - 1)));
                    }
                }
            }
}

static oracle *create_grid(int D, int nx, int ny, int nz, double dx, double dy, double dz, double gamma,
                           double tau, double cfl, double t_end, const int *bc6, const double *inflow,
                           const int *inflow_range, int limiter_kind, double tol, int max_iter,
                           int fixed_iters)
{
    if (D < 1 || D > 3 || nx < 1) return NULL;
    if (D < 2) ny = 1;
    if (D < 3) nz = 1;
    if (ny < 1 || nz < 1) return NULL;
    oracle *o = (oracle *)calloc(1, sizeof(oracle));
    lattice_init(&o->L, D);
    o->D = D; o->Q = o->L.Q; o->nx = nx; o->ny = ny; o->nz = nz;
    o->gx = NG; o->gy = D >= 2 ? NG : 0; o->gz = D == 3 ? NG : 0;
    o->px = nx + 2 * o->gx; o->py = ny + 2 * o->gy; o->pz = nz + 2 * o->gz;
    o->dx = dx; o->dy = D >= 2 ? dy : 1.0; o->dz = D == 3 ? dz : 1.0;
    o->gamma = gamma; o->Cv = 1.0 / (gamma - 1.0);
    o->tau = tau; o->cfl = cfl; o->t_end = t_end;
    for (int s = 0; s < 6; ++s) o->bc[s] = bc6 ? bc6[s] : BC_TRANSMISSIVE;
    for (int s = 0; s < 4; ++s) {
        for (int q = 0; q < 4; ++q) o->inflow[s][q] = inflow ? inflow[s * 4 + q] : 0.0;
        o->inflow_lo[s] = inflow_range ? inflow_range[2 * s] : 0;
        o->inflow_hi[s] = inflow_range ? inflow_range[2 * s + 1] : 0;
    }
    o->limiter = limiter_kind; o->tol = tol; o->max_iter = max_iter; o->fixed_iters = fixed_iters;
    size_t nc = (size_t)o->px * o->py * o->pz;
    o->f = calloc(nc * o->Q, sizeof(double));
    o->g = calloc(nc * o->Q, sizeof(double));
    o->fp = calloc(nc * o->Q, sizeof(double));
    o->gp = calloc(nc * o->Q, sizeof(double));
    o->u = calloc(nc * MAXD, sizeof(double));
    o->T = calloc(nc, sizeof(double));
    o->un = calloc(nc * MAXD, sizeof(double));
    o->Tn = calloc(nc, sizeof(double));
    size_t nxf = (size_t)(nx + 1) * ny * nz, nyf = (size_t)nx * (ny + 1) * nz, nzf = (size_t)nx * ny * (nz + 1);
    o->xu = calloc(nxf * MAXD, sizeof(double)); o->xT = calloc(nxf, sizeof(double));
    o->xf = calloc(nxf * o->Q, sizeof(double)); o->xg = calloc(nxf * o->Q, sizeof(double));
    o->yu = calloc(nyf * MAXD, sizeof(double)); o->yT = calloc(nyf, sizeof(double));
    o->yf = calloc(nyf * o->Q, sizeof(double)); o->yg = calloc(nyf * o->Q, sizeof(double));
    o->zu = calloc(nzf * MAXD, sizeof(double)); o->zT = calloc(nzf, sizeof(double));
    o->zf = calloc(nzf * o->Q, sizeof(double)); o->zg = calloc(nzf * o->Q, sizeof(double));
    return o;
}

oracle *oracle_create(int D, int nx, int ny, double dx, double dy, double gamma, double tau,
                      double cfl, double t_end, const int *bc, const double *inflow,
                      const int *inflow_range, int limiter_kind, double tol, int max_iter,
                      int fixed_iters)
{
    if (D != 1 && D != 2) return NULL;
    int bc6[6] = {BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE};
    for (int s = 0; s < 4; ++s) bc6[s] = bc ? bc[s] : BC_TRANSMISSIVE;
    return create_grid(D, nx, ny, 1, dx, dy, 1.0, gamma, tau, cfl, t_end, bc6, inflow, inflow_range,
                       limiter_kind, tol, max_iter, fixed_iters);
}

/* A D3Q64 grid of nx x ny x nz cells; bc lists x-lo, x-hi, y-lo, y-hi, z-lo, z-hi
 * (transmissive, periodic or reflective; no inflow sides in 3D). */
oracle *oracle_create3(int nx, int ny, int nz, double dx, double dy, double dz, double gamma, double tau,
                       double cfl, double t_end, const int *bc6, int limiter_kind, double tol, int max_iter,
                       int fixed_iters)
{
    for (int s = 0; s < 6; ++s)
        if (bc6 && bc6[s] == BC_INFLOW) return NULL;
    return create_grid(3, nx, ny, nz, dx, dy, dz, gamma, tau, cfl, t_end, bc6, NULL, NULL, limiter_kind,
                       tol, max_iter, fixed_iters);
}

void oracle_free(oracle *o)
{
    if (!o) return;
    free(o->f); free(o->g); free(o->fp); free(o->gp); free(o->u); free(o->T); free(o->un); free(o->Tn);
    free(o->xu); free(o->xT); free(o->xf); free(o->xg);
    free(o->yu); free(o->yT); free(o->yf); free(o->yg);
    free(o->zu); free(o->zT); free(o->zf); free(o->zg);
    free(o);
}

/* Face predictor before the first step: the frame of the pooled conserved moments of the
 * two adjacent cells (their mean density, momentum and total energy). */
static void pooled_frame(const oracle *o, int A, int B, double *u, double *T)
{
    double rA, rB, mA[MAXD] = {0}, mB[MAXD] = {0}, eA, eB, m[MAXD] = {0};
    conserved_moments(&o->L, o->f + (size_t)A * o->Q, o->g + (size_t)A * o->Q, o->u + (size_t)A * MAXD, o->T[A], &rA, mA, &eA);
    conserved_moments(&o->L, o->f + (size_t)B * o->Q, o->g + (size_t)B * o->Q, o->u + (size_t)B * MAXD, o->T[B], &rB, mB, &eB);
    double r = 0.5 * (rA + rB), e = 0.5 * (eA + eB);
    for (int a = 0; a < o->D; ++a) { m[a] = 0.5 * (mA[a] + mB[a]); u[a] = m[a] / r; }
    *T = temperature_from(r, m, e, o->D, o->Cv);
}

/* Frame of the pooled conserved moments of n cells. */
static void pooled_frame_n(const oracle *o, const int *cells, int n, double *u, double *T)
{
    double r = 0.0, m[MAXD] = {0}, e = 0.0;
    for (int s = 0; s < n; ++s) {
        int A = cells[s];
        double rA, mA[MAXD] = {0}, eA;
        conserved_moments(&o->L, o->f + (size_t)A * o->Q, o->g + (size_t)A * o->Q, o->u + (size_t)A * MAXD, o->T[A], &rA, mA, &eA);
        r += rA / n; e += eA / n;
        for (int a = 0; a < o->D; ++a) m[a] += mA[a] / n;
    }
    for (int a = 0; a < o->D; ++a) u[a] = m[a] / r;
    *T = temperature_from(r, m, e, o->D, o->Cv);
}

static void init_face_gauges(oracle *o)
{
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i <= o->nx; ++i) {
                int fidx = xface3(o, i, j, k);
                pooled_frame(o, cidx3(o, i - 1, j, k), cidx3(o, i, j, k), o->xu + (size_t)fidx * MAXD, o->xT + fidx);
            }
    if (o->D < 2) return;
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j <= o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int fidx = yface3(o, i, j, k);
                pooled_frame(o, cidx3(o, i, j - 1, k), cidx3(o, i, j, k), o->yu + (size_t)fidx * MAXD, o->yT + fidx);
            }
    if (o->D < 3) return;
    for (int k = 0; k <= o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int fidx = zface3(o, i, j, k);
                pooled_frame(o, cidx3(o, i, j, k - 1), cidx3(o, i, j, k), o->zu + (size_t)fidx * MAXD, o->zT + fidx);
            }
}

/* Initial condition: equilibrium populations in each cell's co-moving frame, from
 * primitive fields (rho, ux, uy, uz, p) of size nx*ny*nz (x fastest, then y).  uy may be
 * NULL in 1D, uz outside 3D. */
void oracle_set_primitive3(oracle *o, const double *rho, const double *ux, const double *uy,
                           const double *uz, const double *p)
{
    for (int kz = 0; kz < o->nz; ++kz)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int k = (kz * o->ny + j) * o->nx + i;
                double uu[3] = {ux[k], (o->D >= 2 && uy) ? uy[k] : 0.0, (o->D == 3 && uz) ? uz[k] : 0.0};
                set_equilibrium_cell(o, cidx3(o, i, j, kz), rho[k], uu, p[k]);
            }
    fill_ghosts(o);
    init_face_gauges(o);
    o->t = 0.0; o->dt = 0.0; o->steps = 0;
    o->face_iters = o->face_count = o->nonconv = o->nonphys = o->fallbacks = 0;
}

void oracle_set_primitive(oracle *o, const double *rho, const double *ux, const double *uy,
                          const double *p)
{
    oracle_set_primitive3(o, rho, ux, uy, NULL, p);
}

static int bad(double x) { return !(x == x) || isinf(x); }

/* Algorithm step 1: express the populations of a cell in its own co-moving frame. */
static void regauge_cell(oracle *o, int c)
{
    const lattice *L = &o->L;
    double *f = o->f + (size_t)c * o->Q, *g = o->g + (size_t)c * o->Q;
    double *u = o->u + (size_t)c * MAXD;
    double rho, mom[MAXD] = {0}, rhoE;
    conserved_moments(L, f, g, u, o->T[c], &rho, mom, &rhoE);
    double un[MAXD] = {0};
    for (int a = 0; a < o->D; ++a) un[a] = mom[a] / rho;
    double Tn = temperature_from(rho, mom, rhoE, o->D, o->Cv);
    if (!(rho > 0.0) || !(Tn > 0.0) || bad(rho) || bad(Tn)) { o->nonphys++; return; }
    double fo[MAXQ], go[MAXQ];
    grad_transform(L, 3, f, u, o->T[c], un, Tn, fo);
    grad_transform(L, 2, g, u, o->T[c], un, Tn, go);
    memcpy(f, fo, sizeof(double) * o->Q);
    memcpy(g, go, sizeof(double) * o->Q);
    for (int a = 0; a < o->D; ++a) u[a] = un[a];
    o->T[c] = Tn;
}

/* CFL = max|v_ia| dt/dx with v_i = sqrt(T/T_L) c_i + u over all interior cells. */
static double cfl_dt(const oracle *o)
{
    double cmax = 0.0;
    for (int i = 0; i < o->Q; ++i)
        for (int a = 0; a < o->D; ++a) cmax = fmax(cmax, fabs(o->L.c[i][a]));
    double rate = 0.0;
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int c = cidx3(o, i, j, k);
                double s = sqrt(o->T[c] / o->L.TL) * cmax;
                rate = fmax(rate, (fabs(o->u[(size_t)c * MAXD + 0]) + s) / o->dx);
                if (o->D >= 2) rate = fmax(rate, (fabs(o->u[(size_t)c * MAXD + 1]) + s) / o->dy);
                if (o->D == 3) rate = fmax(rate, (fabs(o->u[(size_t)c * MAXD + 2]) + s) / o->dz);
            }
    return o->cfl / rate;
}

/* One face (Sec. III.B.3).  dir = 0: x-face, 1: y-face, 2: z-face.  Cells along the
 * normal: LL, L, R, RR; neighbours of L and R along the first tangential axis (the other
 * axes in increasing order): Lm, Lp, Rm, Rp (2D and 3D); along the second (3D): Lm2, Lp2,
 * Rm2, Rp2.  Writes the face gauge (in/out) and the face populations phi (in the face
 * frame). */
static void solve_face(oracle *o, int dir, const int *cells, double *gu, double *gT,
                       double *face_f, double *face_g, double h)
{
    const lattice *L = &o->L;
    const int D = o->D, Q = o->Q;
    const double sp[3] = {o->dx, o->dy, o->dz};
    const double dn = sp[dir];                    /* spacing along the normal */
    const int tdir = dir == 0 ? 1 : 0;            /* first tangential axis */
    const int tdir2 = dir == 2 ? 1 : 2;           /* second tangential axis (3D) */
    const double dtg = sp[tdir], dtg2 = sp[tdir2];
    const int ncell = D == 3 ? 12 : (D == 2 ? 8 : 4);
    double pf[12][MAXQ], pg[12][MAXQ];
    double lam_u[MAXD] = {0}, lam_T = *gT;
    for (int a = 0; a < D; ++a) lam_u[a] = gu[a];
    double fbar[MAXQ], gbar[MAXQ];
    /* the last pass that defined a frame: its populations, the frame it ran in, its moments */
    double keep_f[MAXQ], keep_g[MAXQ], keep_in_u[MAXD] = {0}, keep_in_T = 0.0;
    double keep_u[MAXD] = {0}, keep_T = 0.0, keep_rho = 0.0;
    int have = 0, iters = 0, done = 0, restarted = 0;
    for (int k = 0; k < o->max_iter && !done; ++k) {
        /* regularized transformation of phi-bar-plus of every stencil cell into lambda_k */
        for (int s = 0; s < ncell; ++s) {
            int c = cells[s];
            grad_transform(L, 3, o->fp + (size_t)c * Q, o->u + (size_t)c * MAXD, o->T[c], lam_u, lam_T, pf[s]);
            grad_transform(L, 2, o->gp + (size_t)c * Q, o->u + (size_t)c * MAXD, o->T[c], lam_u, lam_T, pg[s]);
        }
        double sq = sqrt(lam_T / L->TL);
        for (int i = 0; i < Q; ++i) {
            double v[MAXD];
            for (int a = 0; a < D; ++a) v[a] = sq * L->c[i][a] + lam_u[a];
            /* upwind cell and its neighbours: [upstream, up, downstream, tangential-, tangential+] */
            int up, lo, hi, tm, tp;
            double off_n;
            if (v[dir] > 0.0) { up = 1; lo = 0; hi = 2; tm = 4; tp = 5; off_n = 0.5 * dn; }
            else              { up = 2; lo = 1; hi = 3; tm = 6; tp = 7; off_n = -0.5 * dn; }
            /* departure point x' = x_b - v h, measured from the upwind cell centre */
            double dxn = off_n - v[dir] * h;
            double dxt = D >= 2 ? -v[tdir] * h : 0.0;
            double dxt2 = D == 3 ? -v[tdir2] * h : 0.0;
            for (int pop = 0; pop < 2; ++pop) {
                double (*P)[MAXQ] = pop == 0 ? pf : pg;
                double sn = limiter(o->limiter, (P[up][i] - P[lo][i]) / dn, (P[hi][i] - P[up][i]) / dn);
                double st = 0.0;
                if (D >= 2)
                    st = limiter(o->limiter, (P[up][i] - P[tm][i]) / dtg, (P[tp][i] - P[up][i]) / dtg);
                double val = P[up][i] + dxn * sn + dxt * st;
                if (D == 3) {
                    /* the second tangential neighbours sit 4 slots after the first */
                    double st2 = limiter(o->limiter, (P[up][i] - P[tm + 4][i]) / dtg2, (P[tp + 4][i] - P[up][i]) / dtg2);
                    val += dxt2 * st2;
                }
                if (pop == 0) fbar[i] = val; else gbar[i] = val;
            }
        }
        /* Eqs. (correctorfieldsrhoDUGKS)-(correctorfieldsTDUGKS) */
        double rho1, mom[MAXD] = {0}, rhoE, u1[MAXD] = {0};
        conserved_moments(L, fbar, gbar, lam_u, lam_T, &rho1, mom, &rhoE);
        for (int a = 0; a < D; ++a) u1[a] = mom[a] / rho1;
        double T1 = temperature_from(rho1, mom, rhoE, D, o->Cv);
        iters = k + 1;
        if (!(T1 > 0.0) || bad(rho1) || bad(T1) || bad(u1[0]) || (D >= 2 && bad(u1[1])) || (D == 3 && bad(u1[2]))) {
            /* this pass defines no frame: restart once from the pooled frame of the whole
             * face stencil, otherwise stop at the last pass that did */
            o->fallbacks++;
            if (!restarted) {
                restarted = 1;
                pooled_frame_n(o, cells, ncell, lam_u, &lam_T);
                continue;
            }
            break;
        }
        memcpy(keep_f, fbar, sizeof(keep_f));
        memcpy(keep_g, gbar, sizeof(keep_g));
        for (int a = 0; a < D; ++a) { keep_in_u[a] = lam_u[a]; keep_u[a] = u1[a]; }
        keep_in_T = lam_T; keep_T = T1; keep_rho = rho1;
        have = 1;
        if (o->fixed_iters > 0) {
            done = iters >= o->fixed_iters;
        } else {
            double du = 0.0;
            for (int a = 0; a < D; ++a) du = fmax(du, fabs(u1[a] - lam_u[a]));
            done = du <= o->tol * sqrt(lam_T) && fabs(T1 - lam_T) <= o->tol * lam_T;
        }
        for (int a = 0; a < D; ++a) lam_u[a] = u1[a];
        lam_T = T1;
    }
    o->face_iters += iters;
    o->face_count += 1;
    if (!done) o->nonconv++;
    if (!have) { o->nonphys++; keep_T = NAN; keep_in_T = NAN; }
    /* Eq. (FluxTransf) at the frame defined by the moments of the last valid pass, with the
     * exact co-moving equilibria there: phi = (2 tau phibar + h phi^eq) / (2 tau + h). */
    double fb2[MAXQ], gb2[MAXQ], feq[MAXQ], geq[MAXQ];
    grad_transform(L, 3, keep_f, keep_in_u, keep_in_T, keep_u, keep_T, fb2);
    grad_transform(L, 2, keep_g, keep_in_u, keep_in_T, keep_u, keep_T, gb2);
    equilibria(L, keep_rho, keep_T, o->Cv, feq, geq);
    double tau = o->tau;
    for (int i = 0; i < Q; ++i) {
        face_f[i] = (2.0 * tau * fb2[i] + h * feq[i]) / (2.0 * tau + h);
        face_g[i] = (2.0 * tau * gb2[i] + h * geq[i]) / (2.0 * tau + h);
    }
    for (int a = 0; a < D; ++a) gu[a] = keep_u[a];
    *gT = keep_T;
}

/* Adds the contribution (v_i . n) phi_i^{lambda_j} A/V of one face to the flux F of cell c. */
static void add_face_flux(oracle *o, int c, const double *face_u, double face_T,
                          const double *face_f, const double *face_g, int dir, double sign,
                          double area_over_vol, double *Ff, double *Fg)
{
    const lattice *L = &o->L;
    double pf[MAXQ], pg[MAXQ];
    const double *uc = o->u + (size_t)c * MAXD;
    grad_transform(L, 3, face_f, face_u, face_T, uc, o->T[c], pf);
    grad_transform(L, 2, face_g, face_u, face_T, uc, o->T[c], pg);
    double sq = sqrt(o->T[c] / L->TL);
    for (int i = 0; i < o->Q; ++i) {
        double vn = sign * (sq * L->c[i][dir] + uc[dir]);
        Ff[i] += vn * pf[i] * area_over_vol;
        Fg[i] += vn * pg[i] * area_over_vol;
    }
}

static void stencil_x(const oracle *o, int i, int j, int cells[8])
{
    /* x-face i sits between cells (i-1, j) and (i, j) */
    cells[0] = cidx(o, i - 2, j); cells[1] = cidx(o, i - 1, j);
    cells[2] = cidx(o, i, j);     cells[3] = cidx(o, i + 1, j);
    if (o->D == 2) {
        cells[4] = cidx(o, i - 1, j - 1); cells[5] = cidx(o, i - 1, j + 1);
        cells[6] = cidx(o, i, j - 1);     cells[7] = cidx(o, i, j + 1);
    }
}

static void stencil_y(const oracle *o, int i, int j, int cells[8])
{
    /* y-face j sits between cells (i, j-1) and (i, j) */
    cells[0] = cidx(o, i, j - 2); cells[1] = cidx(o, i, j - 1);
    cells[2] = cidx(o, i, j);     cells[3] = cidx(o, i, j + 1);
    cells[4] = cidx(o, i - 1, j - 1); cells[5] = cidx(o, i + 1, j - 1);
    cells[6] = cidx(o, i - 1, j);     cells[7] = cidx(o, i + 1, j);
}

/* 3D stencil of the face of axis dir whose high-side cell is (i, j, k): along the normal
 * two cells on each side, then the neighbours of L and R along the first and the second
 * tangential axis (the same slots as the 2D stencils). */
static void stencil3(const oracle *o, int dir, int i, int j, int k, int cells[12])
{
    int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    const int *n = e[dir], *t1 = e[dir == 0 ? 1 : 0], *t2 = e[dir == 2 ? 1 : 2];
    for (int s = 0; s < 4; ++s)
        cells[s] = cidx3(o, i + (s - 2) * n[0], j + (s - 2) * n[1], k + (s - 2) * n[2]);
    for (int side = 0; side < 2; ++side) {          /* L (side 0) and R (side 1) */
        int bi = i + (side - 1) * n[0], bj = j + (side - 1) * n[1], bk = k + (side - 1) * n[2];
        cells[4 + 2 * side] = cidx3(o, bi - t1[0], bj - t1[1], bk - t1[2]);
        cells[5 + 2 * side] = cidx3(o, bi + t1[0], bj + t1[1], bk + t1[2]);
        cells[8 + 2 * side] = cidx3(o, bi - t2[0], bj - t2[1], bk - t2[2]);
        cells[9 + 2 * side] = cidx3(o, bi + t2[0], bj + t2[1], bk + t2[2]);
    }
}

static void step3(oracle *o, double dt);

/* Advances n time steps (fewer when t_end > 0 is reached).  Returns the number taken. */
int oracle_step(oracle *o, int n)
{
    const lattice *L = &o->L;
    const int Q = o->Q, D = o->D;
    int taken = 0;
    for (int s = 0; s < n; ++s) {
        if (o->t_end > 0.0 && o->t >= o->t_end) break;
        /* 1. every cell in its local frame */
        for (int k = 0; k < o->nz; ++k)
            for (int j = 0; j < o->ny; ++j)
                for (int i = 0; i < o->nx; ++i) regauge_cell(o, cidx3(o, i, j, k));
        fill_ghosts(o);
        double dt = o->forced_dt > 0.0 ? o->forced_dt : cfl_dt(o);
        if (o->t_end > 0.0 && o->t + dt > o->t_end) dt = o->t_end - o->t;
        if (D == 3) {
            step3(o, dt);
            o->t += dt;
            o->last_dt = dt;
            o->steps++;
            taken++;
            continue;
        }
        const double h = 0.5 * dt, tau = o->tau;
        /* 2a. phi-bar-plus at every cell (ghosts included), Eq. (Fbarplus) with Eq. (variableTransform) */
        const double cp = (2.0 * tau - h) / (2.0 * tau + dt), ce = 3.0 * h / (2.0 * tau + dt);
        for (int c = 0; c < o->px * o->py; ++c) {
            double rho = 0.0;
            for (int i = 0; i < Q; ++i) rho += o->f[(size_t)c * Q + i];
            double feq[MAXQ], geq[MAXQ];
            equilibria(L, rho, o->T[c], o->Cv, feq, geq);
            for (int i = 0; i < Q; ++i) {
                o->fp[(size_t)c * Q + i] = cp * o->f[(size_t)c * Q + i] + ce * feq[i];
                o->gp[(size_t)c * Q + i] = cp * o->g[(size_t)c * Q + i] + ce * geq[i];
            }
        }
        /* 2b. face populations at t_{n+1/2} in the co-moving face frame */
        int cells[8];
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i <= o->nx; ++i) {
                int fi = xface(o, i, j);
                stencil_x(o, i, j, cells);
                solve_face(o, 0, cells, o->xu + (size_t)fi * MAXD, o->xT + fi,
                           o->xf + (size_t)fi * Q, o->xg + (size_t)fi * Q, h);
            }
        if (D == 2)
            for (int j = 0; j <= o->ny; ++j)
                for (int i = 0; i < o->nx; ++i) {
                    int fi = yface(o, i, j);
                    stencil_y(o, i, j, cells);
                    solve_face(o, 1, cells, o->yu + (size_t)fi * MAXD, o->yT + fi,
                               o->yf + (size_t)fi * Q, o->yg + (size_t)fi * Q, h);
                }
        /* 3. flux into each cell's frame, Eq. (fluxEq), and update, Eqs. (FinalUpdateDUGKS) */
        const double ca = (2.0 * tau - dt) / (2.0 * tau + dt), cb = 2.0 * dt / (2.0 * tau + dt);
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int c = cidx(o, i, j);
                double Ff[MAXQ] = {0}, Fg[MAXQ] = {0};
                int fl = xface(o, i, j), fr = xface(o, i + 1, j);
                add_face_flux(o, c, o->xu + (size_t)fl * MAXD, o->xT[fl], o->xf + (size_t)fl * Q,
                              o->xg + (size_t)fl * Q, 0, -1.0, 1.0 / o->dx, Ff, Fg);
                add_face_flux(o, c, o->xu + (size_t)fr * MAXD, o->xT[fr], o->xf + (size_t)fr * Q,
                              o->xg + (size_t)fr * Q, 0, +1.0, 1.0 / o->dx, Ff, Fg);
                if (D == 2) {
                    int fb = yface(o, i, j), ft = yface(o, i, j + 1);
                    add_face_flux(o, c, o->yu + (size_t)fb * MAXD, o->yT[fb], o->yf + (size_t)fb * Q,
                                  o->yg + (size_t)fb * Q, 1, -1.0, 1.0 / o->dy, Ff, Fg);
                    add_face_flux(o, c, o->yu + (size_t)ft * MAXD, o->yT[ft], o->yf + (size_t)ft * Q,
                                  o->yg + (size_t)ft * Q, 1, +1.0, 1.0 / o->dy, Ff, Fg);
                }
                double rho = 0.0;
                for (int q = 0; q < Q; ++q) rho += o->f[(size_t)c * Q + q];
                double feq[MAXQ], geq[MAXQ];
                equilibria(L, rho, o->T[c], o->Cv, feq, geq);
                for (int q = 0; q < Q; ++q) {
                    double *fq = o->f + (size_t)c * Q + q, *gq = o->g + (size_t)c * Q + q;
                    *fq = ca * *fq + cb * feq[q] - dt * Ff[q];
                    *gq = ca * *gq + cb * geq[q] - dt * Fg[q];
                }
            }
        o->t += dt;
        o->last_dt = dt;
        o->steps++;
        taken++;
    }
    return taken;
}

/* Steps 2 and 3 of the algorithm on a D3Q64 grid (the 1D/2D loops above with a third
 * axis): phi-bar-plus everywhere, the faces of the three axes, then the flux of the six
 * faces of every cell and the update. */
static void step3(oracle *o, double dt)
{
    const lattice *L = &o->L;
    const int Q = o->Q;
    const double h = 0.5 * dt, tau = o->tau;
    const double cp = (2.0 * tau - h) / (2.0 * tau + dt), ce = 3.0 * h / (2.0 * tau + dt);
    for (int c = 0; c < o->px * o->py * o->pz; ++c) {
        double rho = 0.0;
        for (int i = 0; i < Q; ++i) rho += o->f[(size_t)c * Q + i];
        double feq[MAXQ], geq[MAXQ];
        equilibria(L, rho, o->T[c], o->Cv, feq, geq);
        for (int i = 0; i < Q; ++i) {
            o->fp[(size_t)c * Q + i] = cp * o->f[(size_t)c * Q + i] + ce * feq[i];
            o->gp[(size_t)c * Q + i] = cp * o->g[(size_t)c * Q + i] + ce * geq[i];
        }
    }
    int cells[12];
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i <= o->nx; ++i) {
                int fi = xface3(o, i, j, k);
                stencil3(o, 0, i, j, k, cells);
                solve_face(o, 0, cells, o->xu + (size_t)fi * MAXD, o->xT + fi, o->xf + (size_t)fi * Q, o->xg + (size_t)fi * Q, h);
            }
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j <= o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int fi = yface3(o, i, j, k);
                stencil3(o, 1, i, j, k, cells);
                solve_face(o, 1, cells, o->yu + (size_t)fi * MAXD, o->yT + fi, o->yf + (size_t)fi * Q, o->yg + (size_t)fi * Q, h);
            }
    for (int k = 0; k <= o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int fi = zface3(o, i, j, k);
                stencil3(o, 2, i, j, k, cells);
                solve_face(o, 2, cells, o->zu + (size_t)fi * MAXD, o->zT + fi, o->zf + (size_t)fi * Q, o->zg + (size_t)fi * Q, h);
            }
    const double ca = (2.0 * tau - dt) / (2.0 * tau + dt), cb = 2.0 * dt / (2.0 * tau + dt);
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int c = cidx3(o, i, j, k);
                double Ff[MAXQ] = {0}, Fg[MAXQ] = {0};
                int fl = xface3(o, i, j, k), fr = xface3(o, i + 1, j, k);
                int fb = yface3(o, i, j, k), ft = yface3(o, i, j + 1, k);
                int fd = zface3(o, i, j, k), fu = zface3(o, i, j, k + 1);
                add_face_flux(o, c, o->xu + (size_t)fl * MAXD, o->xT[fl], o->xf + (size_t)fl * Q, o->xg + (size_t)fl * Q, 0, -1.0, 1.0 / o->dx, Ff, Fg);
                add_face_flux(o, c, o->xu + (size_t)fr * MAXD, o->xT[fr], o->xf + (size_t)fr * Q, o->xg + (size_t)fr * Q, 0, +1.0, 1.0 / o->dx, Ff, Fg);
                add_face_flux(o, c, o->yu + (size_t)fb * MAXD, o->yT[fb], o->yf + (size_t)fb * Q, o->yg + (size_t)fb * Q, 1, -1.0, 1.0 / o->dy, Ff, Fg);
                add_face_flux(o, c, o->yu + (size_t)ft * MAXD, o->yT[ft], o->yf + (size_t)ft * Q, o->yg + (size_t)ft * Q, 1, +1.0, 1.0 / o->dy, Ff, Fg);
                add_face_flux(o, c, o->zu + (size_t)fd * MAXD, o->zT[fd], o->zf + (size_t)fd * Q, o->zg + (size_t)fd * Q, 2, -1.0, 1.0 / o->dz, Ff, Fg);
                add_face_flux(o, c, o->zu + (size_t)fu * MAXD, o->zT[fu], o->zf + (size_t)fu * Q, o->zg + (size_t)fu * Q, 2, +1.0, 1.0 / o->dz, Ff, Fg);
                double rho = 0.0;
                for (int q = 0; q < Q; ++q) rho += o->f[(size_t)c * Q + q];
                double feq[MAXQ], geq[MAXQ];
                equilibria(L, rho, o->T[c], o->Cv, feq, geq);
                for (int q = 0; q < Q; ++q) {
                    double *fq = o->f + (size_t)c * Q + q, *gq = o->g + (size_t)c * Q + q;
                    *fq = ca * *fq + cb * feq[q] - dt * Ff[q];
                    *gq = ca * *gq + cb * geq[q] - dt * Fg[q];
                }
            }
}

/* ------------------------------------------------- semi-Lagrangian realization */

/* Interpolation for the semi-Lagrangian step (Sec. III.A uses a 4-point stencil with a
 * B-spline kernel and limiters whose details are in a thesis that is not available).
 * Reading: the 4-point Lagrange interpolant (exact for cubics) at collocation offsets
 * -1, 0, 1, 2, evaluated at th in [0, 1] (in 2D its tensor product on the 4 x 4 points);
 * if it leaves the interval spanned by the bracketing values (the 2 nearest points, or the
 * 2 x 2 nearest in 2D), the linear (bilinear) interpolant of those values is used. */
static void lagrange4_weights(double th, double *w)
{
    w[0] = -th * (th - 1.0) * (th - 2.0) / 6.0;
    w[1] = (th + 1.0) * (th - 1.0) * (th - 2.0) / 2.0;
    w[2] = -(th + 1.0) * th * (th - 2.0) / 2.0;
    w[3] = (th + 1.0) * th * (th - 1.0) / 6.0;
}

static double sl_interp(const double *v, double th)
{
    double w[4];
    lagrange4_weights(th, w);
    double p = w[0] * v[0] + w[1] * v[1] + w[2] * v[2] + w[3] * v[3];
    const double lo = fmin(v[1], v[2]), hi = fmax(v[1], v[2]);
    if (p < lo || p > hi) p = v[1] + th * (v[2] - v[1]);
    return p;
}

/* v[r][m]: row r along y (offsets -1..2), column m along x */
static double sl_interp2(double v[4][4], double thx, double thy)
{
    double wx[4], wy[4];
    lagrange4_weights(thx, wx);
    lagrange4_weights(thy, wy);
    double p = 0.0;
    for (int r = 0; r < 4; ++r)
        for (int m = 0; m < 4; ++m) p += wy[r] * wx[m] * v[r][m];
    const double lo = fmin(fmin(v[1][1], v[1][2]), fmin(v[2][1], v[2][2]));
    const double hi = fmax(fmax(v[1][1], v[1][2]), fmax(v[2][1], v[2][2]));
    if (p < lo || p > hi)
        p = (1.0 - thy) * ((1.0 - thx) * v[1][1] + thx * v[1][2]) + thy * ((1.0 - thx) * v[2][1] + thx * v[2][2]);
    return p;
}

/* Base collocation point and fraction of a departure point x_node - d along one axis, in
 * units of the spacing: base = node - 1 when d > 0, else node (so |d| < h keeps th in [0, 1]). */
static void sl_base(double d_over_h, int *base_off, double *th)
{
    if (d_over_h > 0.0) { *base_off = -1; *th = 1.0 - d_over_h; }
    else                { *base_off = 0;  *th = -d_over_h; }
}

/* One node of the semi-Lagrangian step (Sec. III.A): predictor-corrector on the node's
 * frame, each pass advecting every population from its departure point x - v_i dt with
 * the stencil re-expressed in the pass's frame (regularized transformation, Sec. II.C),
 * then the BGK collision with beta = dt / (2 tau + dt).  The corrector readings of the
 * finite-volume faces apply unchanged (convergence rule, restart from the pooled moments
 * of the stencil, the last valid pass's moments Grad-projected into the frame they define).
 * Writes the new populations and frame of the node into fp/gp/un/Tn. */
static void sl_node(oracle *o, int i, int j, double dt)
{
    const lattice *L = &o->L;
    const int D = o->D, Q = o->Q;
    const int R = 2, W = 2 * R + 1;              /* stencil i-2..i+2 (and j-2..j+2 in 2D) */
    const int ny_s = D == 2 ? W : 1;
    int cells[25];
    int ns = 0;
    for (int b = 0; b < ny_s; ++b)
        for (int a = 0; a < W; ++a) cells[ns++] = cidx(o, i - R + a, D == 2 ? j - R + b : j);
    const int c0 = cidx(o, i, j);
    double pf[25][MAXQ], pg[25][MAXQ];
    double lam_u[MAXD] = {0}, lam_T = o->T[c0];
    for (int a = 0; a < D; ++a) lam_u[a] = o->u[(size_t)c0 * MAXD + a];
    double fbar[MAXQ], gbar[MAXQ];
    double keep_f[MAXQ], keep_g[MAXQ], keep_in_u[MAXD] = {0}, keep_in_T = 0.0;
    double keep_u[MAXD] = {0}, keep_T = 0.0, keep_rho = 0.0;
    int have = 0, iters = 0, done = 0, restarted = 0;
    for (int k = 0; k < o->max_iter && !done; ++k) {
        for (int s = 0; s < ns; ++s) {
            int c = cells[s];
            grad_transform(L, 3, o->f + (size_t)c * Q, o->u + (size_t)c * MAXD, o->T[c], lam_u, lam_T, pf[s]);
            grad_transform(L, 2, o->g + (size_t)c * Q, o->u + (size_t)c * MAXD, o->T[c], lam_u, lam_T, pg[s]);
        }
        const double sq = sqrt(lam_T / L->TL);
        for (int q = 0; q < Q; ++q) {
            double v[MAXD];
            for (int a = 0; a < D; ++a) v[a] = sq * L->c[q][a] + lam_u[a];
            int bx, by = 0;
            double thx, thy = 0.0;
            sl_base(v[0] * dt / o->dx, &bx, &thx);
            if (D == 2) sl_base(v[1] * dt / o->dy, &by, &thy);
            for (int pop = 0; pop < 2; ++pop) {
                double (*P)[MAXQ] = pop == 0 ? pf : pg;
                double val;
                if (D == 1) {
                    double col[4];
                    for (int m = 0; m < 4; ++m) col[m] = P[R + bx - 1 + m][q];
                    val = sl_interp(col, thx);
                } else {
                    double box[4][4];
                    for (int r = 0; r < 4; ++r)
                        for (int m = 0; m < 4; ++m) box[r][m] = P[(R + by - 1 + r) * W + R + bx - 1 + m][q];
                    val = sl_interp2(box, thx, thy);
                }
                if (pop == 0) fbar[q] = val; else gbar[q] = val;
            }
        }
        /* Eqs. (correctorfieldsrho)-(correctorfieldT) */
        double rho1, mom[MAXD] = {0}, rhoE, u1[MAXD] = {0};
        conserved_moments(L, fbar, gbar, lam_u, lam_T, &rho1, mom, &rhoE);
        for (int a = 0; a < D; ++a) u1[a] = mom[a] / rho1;
        double T1 = temperature_from(rho1, mom, rhoE, D, o->Cv);
        iters = k + 1;
        if (!(T1 > 0.0) || bad(rho1) || bad(T1) || bad(u1[0]) || (D == 2 && bad(u1[1]))) {
            o->fallbacks++;
            if (!restarted) {
                restarted = 1;
                pooled_frame_n(o, cells, ns, lam_u, &lam_T);
                continue;
            }
            break;
        }
        memcpy(keep_f, fbar, sizeof(keep_f));
        memcpy(keep_g, gbar, sizeof(keep_g));
        for (int a = 0; a < D; ++a) { keep_in_u[a] = lam_u[a]; keep_u[a] = u1[a]; }
        keep_in_T = lam_T; keep_T = T1; keep_rho = rho1;
        have = 1;
        if (o->fixed_iters > 0) {
            done = iters >= o->fixed_iters;
        } else {
            double du = 0.0;
            for (int a = 0; a < D; ++a) du = fmax(du, fabs(u1[a] - lam_u[a]));
            done = du <= o->tol * sqrt(lam_T) && fabs(T1 - lam_T) <= o->tol * lam_T;
        }
        for (int a = 0; a < D; ++a) lam_u[a] = u1[a];
        lam_T = T1;
    }
    o->face_iters += iters;
    o->face_count += 1;
    if (!done) o->nonconv++;
    if (!have) { o->nonphys++; keep_T = NAN; keep_in_T = NAN; }
    /* the pre-collision populations in the frame of their own moments, then BGK */
    double fl[MAXQ], gl[MAXQ], feq[MAXQ], geq[MAXQ];
    grad_transform(L, 3, keep_f, keep_in_u, keep_in_T, keep_u, keep_T, fl);
    grad_transform(L, 2, keep_g, keep_in_u, keep_in_T, keep_u, keep_T, gl);
    equilibria(L, keep_rho, keep_T, o->Cv, feq, geq);
    const double beta = dt / (2.0 * o->tau + dt);
    for (int q = 0; q < Q; ++q) {
        o->fp[(size_t)c0 * Q + q] = fl[q] + 2.0 * beta * (feq[q] - fl[q]);
        o->gp[(size_t)c0 * Q + q] = gl[q] + 2.0 * beta * (geq[q] - gl[q]);
    }
    for (int a = 0; a < D; ++a) o->un[(size_t)c0 * MAXD + a] = keep_u[a];
    o->Tn[c0] = keep_T;
}

/* n semi-Lagrangian steps (Sec. III.A); the time step follows the same CFL rule. */
int oracle_sl_step(oracle *o, int n)
{
    const int Q = o->Q, D = o->D;
    int taken = 0;
    if (D == 3) return -1;   /* the semi-Lagrangian step is written for D1Q4 and D2Q16 */
    for (int s = 0; s < n; ++s) {
        if (o->t_end > 0.0 && o->t >= o->t_end) break;
        fill_ghosts(o);
        double dt = o->forced_dt > 0.0 ? o->forced_dt : cfl_dt(o);
        if (o->t_end > 0.0 && o->t + dt > o->t_end) dt = o->t_end - o->t;
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) sl_node(o, i, j, dt);
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int c = cidx(o, i, j);
                memcpy(o->f + (size_t)c * Q, o->fp + (size_t)c * Q, sizeof(double) * Q);
                memcpy(o->g + (size_t)c * Q, o->gp + (size_t)c * Q, sizeof(double) * Q);
                for (int a = 0; a < D; ++a) o->u[(size_t)c * MAXD + a] = o->un[(size_t)c * MAXD + a];
                o->T[c] = o->Tn[c];
            }
        o->t += dt;
        o->last_dt = dt;
        o->steps++;
        taken++;
    }
    return taken;
}

/* --------------------------------------------------------------- read-back */

/* Conserved fields per interior cell (x fastest, then y, then z); my may be NULL in 1D,
 * mz outside 3D. */
void oracle_conserved3(const oracle *o, double *rho, double *mx, double *my, double *mz, double *E)
{
    for (int kz = 0; kz < o->nz; ++kz)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int c = cidx3(o, i, j, kz), k = (kz * o->ny + j) * o->nx + i;
                double r, m[MAXD] = {0}, e;
                conserved_moments(&o->L, o->f + (size_t)c * o->Q, o->g + (size_t)c * o->Q,
                                  o->u + (size_t)c * MAXD, o->T[c], &r, m, &e);
                rho[k] = r; mx[k] = m[0];
                if (my) my[k] = o->D >= 2 ? m[1] : 0.0;
                if (mz) mz[k] = o->D == 3 ? m[2] : 0.0;
                E[k] = e;
            }
}

void oracle_conserved(const oracle *o, double *rho, double *mx, double *my, double *E)
{
    oracle_conserved3(o, rho, mx, my, NULL, E);
}

/* Populations and frames of the interior cells, each first re-expressed in its own
 * co-moving frame (algorithm step 1, on a copy; the stored state is not changed).
 * f, g: [cells][Q]; u: [cells][D]; T: [cells]. */
void oracle_regauged_state(const oracle *o, double *f, double *g, double *u, double *T)
{
    const lattice *L = &o->L;
    for (int kz = 0; kz < o->nz; ++kz)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int c = cidx3(o, i, j, kz), k = (kz * o->ny + j) * o->nx + i;
                const double *fc = o->f + (size_t)c * o->Q, *gc = o->g + (size_t)c * o->Q;
                const double *uc = o->u + (size_t)c * MAXD;
                double rho, mom[MAXD] = {0}, rhoE, un[MAXD] = {0};
                conserved_moments(L, fc, gc, uc, o->T[c], &rho, mom, &rhoE);
                for (int a = 0; a < o->D; ++a) un[a] = mom[a] / rho;
                double Tn = temperature_from(rho, mom, rhoE, o->D, o->Cv);
                grad_transform(L, 3, fc, uc, o->T[c], un, Tn, f + (size_t)k * o->Q);
                grad_transform(L, 2, gc, uc, o->T[c], un, Tn, g + (size_t)k * o->Q);
                for (int a = 0; a < o->D; ++a) u[(size_t)k * o->D + a] = un[a];
                T[k] = Tn;
            }
}

/* Raw state (populations as stored, in the frame of the previous step). */
void oracle_raw_state(const oracle *o, double *f, double *g, double *u, double *T)
{
    for (int kz = 0; kz < o->nz; ++kz)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int c = cidx3(o, i, j, kz), k = (kz * o->ny + j) * o->nx + i;
                memcpy(f + (size_t)k * o->Q, o->f + (size_t)c * o->Q, sizeof(double) * o->Q);
                memcpy(g + (size_t)k * o->Q, o->g + (size_t)c * o->Q, sizeof(double) * o->Q);
                for (int a = 0; a < o->D; ++a) u[(size_t)k * o->D + a] = o->u[(size_t)c * MAXD + a];
                T[k] = o->T[c];
            }
}

/* Overwrites the interior state with populations (f, g) given in frames (u, T). */
void oracle_set_state(oracle *o, const double *f, const double *g, const double *u, const double *T)
{
    for (int kz = 0; kz < o->nz; ++kz)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                int c = cidx3(o, i, j, kz), k = (kz * o->ny + j) * o->nx + i;
                memcpy(o->f + (size_t)c * o->Q, f + (size_t)k * o->Q, sizeof(double) * o->Q);
                memcpy(o->g + (size_t)c * o->Q, g + (size_t)k * o->Q, sizeof(double) * o->Q);
                for (int a = 0; a < o->D; ++a) o->u[(size_t)c * MAXD + a] = u[(size_t)k * o->D + a];
                o->T[c] = T[k];
            }
    fill_ghosts(o);
    init_face_gauges(o);
}

/* Face gauges as (u..., T) rows: x-faces [(nx+1)*ny*nz][D+1], then y-faces
 * [nx*(ny+1)*nz][D+1] (2D, 3D), then z-faces [nx*ny*(nz+1)][D+1] (3D), each x fastest. */
void oracle_face_gauges3(const oracle *o, double *xg, double *yg, double *zg)
{
    int D = o->D;
    const double *us[3] = {o->xu, o->yu, o->zu}, *Ts[3] = {o->xT, o->yT, o->zT};
    double *out[3] = {xg, yg, zg};
    long long nf[3] = {(long long)(o->nx + 1) * o->ny * o->nz, (long long)o->nx * (o->ny + 1) * o->nz,
                       (long long)o->nx * o->ny * (o->nz + 1)};
    for (int d = 0; d < D; ++d) {
        if (!out[d]) continue;
        for (long long k = 0; k < nf[d]; ++k) {
            for (int a = 0; a < D; ++a) out[d][k * (D + 1) + a] = us[d][k * MAXD + a];
            out[d][k * (D + 1) + D] = Ts[d][k];
        }
    }
}

void oracle_face_gauges(const oracle *o, double *xg, double *yg)
{
    oracle_face_gauges3(o, xg, o->D == 2 ? yg : NULL, NULL);
}

/* Overwrites the face gauges (same layout as oracle_face_gauges3). */
void oracle_set_face_gauges3(oracle *o, const double *xg, const double *yg, const double *zg)
{
    int D = o->D;
    double *us[3] = {o->xu, o->yu, o->zu}, *Ts[3] = {o->xT, o->yT, o->zT};
    const double *in[3] = {xg, yg, zg};
    long long nf[3] = {(long long)(o->nx + 1) * o->ny * o->nz, (long long)o->nx * (o->ny + 1) * o->nz,
                       (long long)o->nx * o->ny * (o->nz + 1)};
    for (int d = 0; d < D; ++d) {
        if (!in[d]) continue;
        for (long long k = 0; k < nf[d]; ++k) {
            for (int a = 0; a < D; ++a) us[d][k * MAXD + a] = in[d][k * (D + 1) + a];
            Ts[d][k] = in[d][k * (D + 1) + D];
        }
    }
}

void oracle_set_face_gauges(oracle *o, const double *xg, const double *yg)
{
    oracle_set_face_gauges3(o, xg, o->D == 2 ? yg : NULL, NULL);
}

/* time, last dt, steps, face iterations, faces solved, non-converged faces, non-physical
 * events, corrector passes that defined no frame */
void oracle_stats(const oracle *o, double *t, double *dt, long long *counts)
{
    *t = o->t; *dt = o->last_dt;
    counts[0] = o->steps; counts[1] = o->face_iters; counts[2] = o->face_count;
    counts[3] = o->nonconv; counts[4] = o->nonphys; counts[5] = o->fallbacks;
}

/* ------------------------------------------------ unit-level entry points */

int oracle_lattice(int D, double *c, double *w, double *TL)
{
    lattice L;
    if (D < 1 || D > 3) return 0;
    lattice_init(&L, D);
    for (int i = 0; i < L.Q; ++i) {
        for (int a = 0; a < D; ++a) c[i * D + a] = L.c[i][a];
        w[i] = L.W[i];
    }
    *TL = L.TL;
    return L.Q;
}

void oracle_grad_transform(int D, int order, const double *f_in, const double *u_in, double T_in,
                           const double *u_out, double T_out, double *f_out)
{
    lattice L;
    lattice_init(&L, D);
    grad_transform(&L, order, f_in, u_in, T_in, u_out, T_out, f_out);
}

double oracle_limiter(int kind, double a, double b) { return limiter(kind, a, b); }

/* Test hook: use this time step instead of the CFL one (dt <= 0 restores the CFL rule).
 * Lets a test run one step of a patch cut out of a larger grid with the larger grid's dt. */
void oracle_force_dt(oracle *o, double dt) { o->forced_dt = dt; }

/* Ablation switch: 1 replaces Grad's projection in every regularized transformation by
 * the equilibration of the fast moments (Sec. II.C); 0 restores Grad's. */
void oracle_set_equilibration(oracle *o, int on) { o->L.equilibrate = on != 0; }

/* The regularized transformation alone (test hook), with the equilibration variant. */
void oracle_grad_transform_eq(int D, int order, int equilibrate, const double *f_in, const double *u_in, double T_in,
                              const double *u_out, double T_out, double *f_out)
{
    lattice L;
    lattice_init(&L, D);
    L.equilibrate = equilibrate;
    grad_transform(&L, order, f_in, u_in, T_in, u_out, T_out, f_out);
}
