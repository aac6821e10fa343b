/*
 * lb_oracle.c -- plain CPU oracle for the forced D3Q19 multiple-relaxation-
 * time lattice Boltzmann method with off-lattice singular point forces
 * (Nash, Adhikari & Cates, "Singular forces and point-like colloids in
 * lattice Boltzmann hydrodynamics").
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark are the only callers. It shares no code,
 * table or header with the CUDA library, and it is written to be read
 * against the paper, not to be fast: every quantity is a loop over its
 * definition, the full streamed lattice is materialised, and nothing is
 * fused or reordered.
 *
 * Precision: `real` is double, or long double when compiled with
 * -DORC_LONG_DOUBLE (the self-check build); exported symbols are then
 * prefixed orcl_ instead of orc_.  Build with -ffp-contract=off so that no
 * multiply-add is fused behind the reader's back.
 *
 * What it computes, per time step n (lattice units, dt = dx = 1):
 *   1. F^n(x) = [x fluid] (g + f_c) + sum_a f_a delta^P(x - R_a^n)
 *      -- Sec. III, regularised point forces, Eq. (deltadef), h = 1.
 *   2. pull streaming  df_i(x, n) = df*_i(x - c_i, n - 1)     -- Sec. II,
 *      propagation step; halfway bounce-back df_i(x) = df*_ibar(x) where
 *      x - c_i is a solid node (walls are not in the paper; a stated
 *      extension for the wall-bounded channel).
 *   3. rho = 1 + sum_i df_i,  rho v = sum_i df_i c_i + F/2     -- Eq.
 *      (macrovariables2).
 *   4. colloids: v(R_s) = sum_r v(r) delta^P(R_s - r), then
 *      R_s += v(R_s) + F_s (1/a - 1/a_L) / (6 pi eta)  -- Sec. IV, the
 *      Faxen update with the a_L subtraction (Eq. a_Ldefn), forward Euler.
 *   5. collision in moment space with ghost modes projected out
 *      -- Eq. (fiexp) with its A and B:
 *        A = sum df c + F
 *        B = S - w_s dev(S - rho vv - tau_s (vF + Fv))
 *              - (w_b/3) tr(S - rho vv - tau_b (vF + Fv)) I,
 *        w = 1/(tau + 1/2),  S = sum df Q
 *      df*_i = w_i [drho + A.c_i / cs^2 + B:Q_i / (2 cs^4)].
 *      B is the reading of the paper's stress update that follows from
 *      Eq. (mrtlbe) with stress eigenvalue 1/tau (the printed sign of the
 *      relaxation term is garbled); the trace is relaxed with its own time
 *      tau_b, which reduces to the paper's single-rate operator when
 *      tau_b = tau_s.
 * The state carried is df = fbar - w_i rho0 with rho0 = 1, the auxiliary
 * distribution of Eq. (transformf) minus the rest-state equilibrium, so that
 * small velocities are not lost to rounding against w_i.
 *
 * Force convention: F is a force density per lattice site, so A = j + F
 * and rho v = j + F/2 (Sec. III/IV use F this way).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORC_LONG_DOUBLE
typedef long double real;
#define R_SQRT sqrtl
#define R_FLOOR floorl
#define SYM(name) orcl_##name
#else
typedef double real;
#define R_SQRT sqrt
#define R_FLOOR floor
#define SYM(name) orc_##name
#endif

#define NQ 19

/* D3Q19 velocity set and weights (Qian et al. 1992; the paper names the
 * DdQn family in Sec. II but does not print the vectors).  Order: rest,
 * the six axis vectors, then the twelve face diagonals; i and i+1 are
 * opposite for odd i. */
static const int CV[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
};

static real weight(int i)
{
    int s = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
    if (s == 0) return (real)1 / (real)3;
    if (s == 1) return (real)1 / (real)18;
    return (real)1 / (real)36;
}

static const real CS2 = (real)1 / (real)3; /* speed of sound squared */

static int opposite(int i)
{
    for (int k = 0; k < NQ; ++k)
        if (CV[k][0] == -CV[i][0] && CV[k][1] == -CV[i][1] && CV[k][2] == -CV[i][2])
            return k;
    return -1;
}

/* Q_i,ab = c_ia c_ib - cs^2 delta_ab  (Sec. II, after Eq. eqf) */
static real Qten(int i, int a, int b)
{
    return (real)(CV[i][a] * CV[i][b]) - (a == b ? CS2 : (real)0);
}

/* ---------------------------------------------------------------- tables */

void SYM(lattice)(int *c, real *w)
{
    for (int i = 0; i < NQ; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = CV[i][a];
        w[i] = weight(i);
    }
}

/* ------------------------------------------------ Peskin kernel, Eq. deltadef */

real SYM(phi)(real r)
{
    real s = r < 0 ? -r : r;
    if (s <= 1) return ((real)3 - 2 * s + R_SQRT((real)1 + 4 * s - 4 * s * s)) / 8;
    if (s <= 2) return ((real)5 - 2 * s - R_SQRT((real)-7 + 12 * s - 4 * s * s)) / 8;
    return 0;
}

/* --------------------------------------------------- one-site collision */

/* Moments of the physical distribution from the auxiliary one,
 * Eq. (macrovariables2): rho = 1 + sum df, rho v = sum df c + F/2. */
void SYM(macro_site)(const real *df, const real *F, real *rho, real *v)
{
    real drho = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < NQ; ++i) {
        drho += df[i];
        for (int a = 0; a < 3; ++a) j[a] += df[i] * CV[i][a];
    }
    *rho = 1 + drho;
    for (int a = 0; a < 3; ++a) v[a] = (j[a] + F[a] / 2) / *rho;
}

/* Post-collision auxiliary distribution, Eq. (fiexp) with A and B as in the
 * file header (shear rate 1/(tau_s + 1/2) on the traceless stress, bulk
 * rate 1/(tau_b + 1/2) on its trace, ghosts projected out). */
void SYM(collide_site)(const real *df, const real *F, real tau_s, real tau_b, real *out)
{
    real drho = 0, j[3] = {0, 0, 0}, S[3][3] = {{0}};
    for (int i = 0; i < NQ; ++i) {
        drho += df[i];
        for (int a = 0; a < 3; ++a) {
            j[a] += df[i] * CV[i][a];
            for (int b = 0; b < 3; ++b) S[a][b] += df[i] * Qten(i, a, b);
        }
    }
    real rho = 1 + drho;
    real v[3];
    for (int a = 0; a < 3; ++a) v[a] = (j[a] + F[a] / 2) / rho;

    real ws = 1 / (tau_s + (real)0.5);
    real wb = 1 / (tau_b + (real)0.5);

    real X[3][3], Y[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            X[a][b] = S[a][b] - rho * v[a] * v[b];
            Y[a][b] = v[a] * F[b] + F[a] * v[b];
        }
    real trX = X[0][0] + X[1][1] + X[2][2];
    real trY = Y[0][0] + Y[1][1] + Y[2][2];

    real A[3], B[3][3];
    for (int a = 0; a < 3; ++a) A[a] = j[a] + F[a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            real d = (a == b) ? 1 : 0;
            real dev = (X[a][b] - tau_s * Y[a][b]) - d * (trX - tau_s * trY) / 3;
            real iso = d * (trX - tau_b * trY) / 3;
            B[a][b] = S[a][b] - ws * dev - wb * iso;
        }

    for (int i = 0; i < NQ; ++i) {
        real ac = 0, bq = 0;
        for (int a = 0; a < 3; ++a) {
            ac += A[a] * CV[i][a];
            for (int b = 0; b < 3; ++b) bq += B[a][b] * Qten(i, a, b);
        }
        out[i] = weight(i) * (drho + ac / CS2 + bq / (2 * CS2 * CS2));
    }
}

/* ------------------------------------------------------- whole lattice */

typedef struct {
    int n[3];         /* lattice nx, ny, nz */
    real tau_s;       /* shear relaxation time: eta = rho cs^2 tau_s */
    real tau_b;       /* bulk relaxation time */
    real g[3];        /* uniform body-force density on fluid nodes */
    real fc[3];       /* uniform extra force density on fluid nodes (counter-force) */
    int wall_lo;      /* solid z-plane index, or -1 */
    int wall_hi;      /* solid z-plane index, or -1 */
    real a_L;         /* lattice offset parameter of the colloid update */
} orc_params;

static long site(const orc_params *p, int x, int y, int z)
{
    return ((long)z * p->n[1] + y) * p->n[0] + x;
}

static int wrapi(int k, int n)
{
    int r = k % n;
    return r < 0 ? r + n : r;
}

static int is_solid(const orc_params *p, int z)
{
    return z == p->wall_lo || z == p->wall_hi;
}

/* Position wrapped into [0, n). */
static real wrapr(real X, int n)
{
    real r = X - (real)n * R_FLOOR(X / (real)n);
    if (r >= (real)n) r = 0;
    if (r < 0) r = 0;
    return r;
}

/* The 4 stencil nodes along one axis and their weights phi(node - X):
 * nodes floor(X)-1 .. floor(X)+2 (Sec. III, support |r| < 2). */
static void stencil_1d(real X, int *node, real *wt)
{
    int b = (int)R_FLOOR(X) - 1;
    for (int k = 0; k < 4; ++k) {
        node[k] = b + k;
        wt[k] = SYM(phi)((real)(b + k) - X);
    }
}

/* F(x) = [fluid](g + fc) + sum_a f_a delta^P(x - R_a)  (Sec. III). */
void SYM(force_field)(const orc_params *p, int npts, const real *pos, const real *f, real *F)
{
    long V = (long)p->n[0] * p->n[1] * p->n[2];
    for (int z = 0; z < p->n[2]; ++z)
        for (int y = 0; y < p->n[1]; ++y)
            for (int x = 0; x < p->n[0]; ++x) {
                long s = site(p, x, y, z);
                for (int a = 0; a < 3; ++a)
                    F[a * V + s] = is_solid(p, z) ? 0 : p->g[a] + p->fc[a];
            }
    for (int s = 0; s < npts; ++s) {
        int nd[3][4];
        real wt[3][4];
        for (int a = 0; a < 3; ++a) stencil_1d(wrapr(pos[3 * s + a], p->n[a]), nd[a], wt[a]);
        for (int k = 0; k < 4; ++k)
            for (int jj = 0; jj < 4; ++jj)
                for (int ii = 0; ii < 4; ++ii) {
                    int x = wrapi(nd[0][ii], p->n[0]);
                    int y = wrapi(nd[1][jj], p->n[1]);
                    int z = wrapi(nd[2][k], p->n[2]);
                    if (is_solid(p, z)) continue;
                    real w = wt[0][ii] * wt[1][jj] * wt[2][k];
                    long q = site(p, x, y, z);
                    for (int a = 0; a < 3; ++a) F[a * V + q] += f[3 * s + a] * w;
                }
    }
}

/* Pull streaming: fs_i(x) = post_i(x - c_i), bounce-back at solid nodes. */
static void stream(const orc_params *p, const real *post, real *fs)
{
    long V = (long)p->n[0] * p->n[1] * p->n[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->n[2]; ++z)
        for (int y = 0; y < p->n[1]; ++y)
            for (int x = 0; x < p->n[0]; ++x) {
                long s = site(p, x, y, z);
                for (int i = 0; i < NQ; ++i) {
                    if (is_solid(p, z)) {
                        fs[i * V + s] = 0;
                        continue;
                    }
                    int xs = wrapi(x - CV[i][0], p->n[0]);
                    int ys = wrapi(y - CV[i][1], p->n[1]);
                    int zs = wrapi(z - CV[i][2], p->n[2]);
                    if (is_solid(p, zs))
                        fs[i * V + s] = post[opposite(i) * V + s];
                    else
                        fs[i * V + s] = post[i * V + site(p, xs, ys, zs)];
                }
            }
}

/* rho and v at every site from a streamed lattice and a force field. */
static void macro_field(const orc_params *p, const real *fs, const real *F, real *rho, real *u)
{
    long V = (long)p->n[0] * p->n[1] * p->n[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->n[2]; ++z)
        for (int y = 0; y < p->n[1]; ++y)
            for (int x = 0; x < p->n[0]; ++x) {
                long s = site(p, x, y, z);
                if (is_solid(p, z)) {
                    rho[s] = 1;
                    for (int a = 0; a < 3; ++a) u[a * V + s] = 0;
                    continue;
                }
                real d[NQ], Fs[3], r, v[3];
                for (int i = 0; i < NQ; ++i) d[i] = fs[i * V + s];
                for (int a = 0; a < 3; ++a) Fs[a] = F[a * V + s];
                SYM(macro_site)(d, Fs, &r, v);
                rho[s] = r;
                for (int a = 0; a < 3; ++a) u[a * V + s] = v[a];
            }
}

/* v(R) = sum over the 64 stencil nodes of v(node) delta^P(R - node). */
static void interp(const orc_params *p, const real *u, const real *R, real *out)
{
    long V = (long)p->n[0] * p->n[1] * p->n[2];
    int nd[3][4];
    real wt[3][4];
    for (int a = 0; a < 3; ++a) stencil_1d(wrapr(R[a], p->n[a]), nd[a], wt[a]);
    for (int a = 0; a < 3; ++a) out[a] = 0;
    for (int k = 0; k < 4; ++k)
        for (int jj = 0; jj < 4; ++jj)
            for (int ii = 0; ii < 4; ++ii) {
                long q = site(p, wrapi(nd[0][ii], p->n[0]), wrapi(nd[1][jj], p->n[1]),
                              wrapi(nd[2][k], p->n[2]));
                real w = wt[0][ii] * wt[1][jj] * wt[2][k];
                for (int a = 0; a < 3; ++a) out[a] += u[a * V + q] * w;
            }
}

/* Advance `nsteps` time steps.  df (19*V, SoA df[i*V + site]) holds the
 * post-collision state df* on entry and on exit.  Points: pos/f are 3*npts
 * (xyz interleaved); points with mobile[s] != 0 are colloids of radius
 * radius[s] and move; the others are fixed.
 * ycorr (3*npts, or NULL): the learned correction of the colloid velocity
 * in units of v0 = |f_s| / (6 pi eta a_s); a colloid then moves by its
 * Sec. IV velocity plus ycorr_s v0.  The correction is a function of the
 * positions at the start of the step, so with ycorr the call advances one
 * step (nsteps must be 1).  Not part of the paper.
 * Returns 0, -1 on allocation failure, -2 for ycorr with nsteps != 1. */
int SYM(run)(const orc_params *p, real *df, int npts, real *pos, const real *f,
             const int *mobile, const real *radius, const real *ycorr, int nsteps)
{
    if (ycorr && nsteps != 1) return -2;
    long V = (long)p->n[0] * p->n[1] * p->n[2];
    real *fs = malloc(sizeof(real) * NQ * V);
    real *F = malloc(sizeof(real) * 3 * V);
    real *rho = malloc(sizeof(real) * V);
    real *u = malloc(sizeof(real) * 3 * V);
    if (!fs || !F || !rho || !u) {
        free(fs); free(F); free(rho); free(u);
        return -1;
    }
    const real pi = (real)3.14159265358979323846264338327950288L;
    real eta = CS2 * p->tau_s; /* eta = rho0 cs^2 tau_s, rho0 = 1 */

    for (int n = 0; n < nsteps; ++n) {
        SYM(force_field)(p, npts, pos, f, F);   /* 1 */
        stream(p, df, fs);                      /* 2 */
        macro_field(p, fs, F, rho, u);          /* 3 */
        for (int s = 0; s < npts; ++s) {        /* 4 */
            if (!mobile[s]) continue;
            real vR[3];
            interp(p, u, &pos[3 * s], vR);
            real c = (1 / radius[s] - 1 / p->a_L) / (6 * pi * eta);
            real v0 = 0; /* velocity unit of the learned correction */
            if (ycorr) {
                real fn = R_SQRT(f[3 * s] * f[3 * s] + f[3 * s + 1] * f[3 * s + 1] + f[3 * s + 2] * f[3 * s + 2]);
                v0 = fn / (6 * pi * eta * radius[s]);
            }
            for (int a = 0; a < 3; ++a) {
                real X = pos[3 * s + a] + vR[a] + f[3 * s + a] * c;
                if (ycorr) X += ycorr[3 * s + a] * v0;
                pos[3 * s + a] = wrapr(X, p->n[a]);
            }
        }
#pragma omp parallel for schedule(static)       /* 5 */
        for (int z = 0; z < p->n[2]; ++z)
            for (int y = 0; y < p->n[1]; ++y)
                for (int x = 0; x < p->n[0]; ++x) {
                    long s = site(p, x, y, z);
                    real d[NQ], Fs[3], o[NQ];
                    if (is_solid(p, z)) {
                        for (int i = 0; i < NQ; ++i) df[i * V + s] = 0;
                        continue;
                    }
                    for (int i = 0; i < NQ; ++i) d[i] = fs[i * V + s];
                    for (int a = 0; a < 3; ++a) Fs[a] = F[a * V + s];
                    SYM(collide_site)(d, Fs, p->tau_s, p->tau_b, o);
                    for (int i = 0; i < NQ; ++i) df[i * V + s] = o[i];
                }
    }
    free(fs); free(F); free(rho); free(u);
    return 0;
}

/* Observables of the state at the current time: rho (V) and u (3*V, SoA)
 * at every site, the velocity interpolated at nq query points, and the
 * totals M = sum rho, P = sum rho v over fluid sites (accumulated in site
 * order).  Any output pointer may be NULL. */
int SYM(observe)(const orc_params *p, const real *df, int npts, const real *pos, const real *f,
                 real *rho_out, real *u_out, int nq, const real *qpos, real *qv, real *totals)
{
    long V = (long)p->n[0] * p->n[1] * p->n[2];
    real *fs = malloc(sizeof(real) * NQ * V);
    real *F = malloc(sizeof(real) * 3 * V);
    real *rho = malloc(sizeof(real) * V);
    real *u = malloc(sizeof(real) * 3 * V);
    if (!fs || !F || !rho || !u) {
        free(fs); free(F); free(rho); free(u);
        return -1;
    }
    SYM(force_field)(p, npts, pos, f, F);
    stream(p, df, fs);
    macro_field(p, fs, F, rho, u);
    if (rho_out) memcpy(rho_out, rho, sizeof(real) * V);
    if (u_out) memcpy(u_out, u, sizeof(real) * 3 * V);
    for (int s = 0; s < nq; ++s) interp(p, u, &qpos[3 * s], &qv[3 * s]);
    if (totals) {
        for (int a = 0; a < 4; ++a) totals[a] = 0;
        for (int z = 0; z < p->n[2]; ++z) {
            if (is_solid(p, z)) continue;
            for (int y = 0; y < p->n[1]; ++y)
                for (int x = 0; x < p->n[0]; ++x) {
                    long s = site(p, x, y, z);
                    totals[0] += rho[s];
                    for (int a = 0; a < 3; ++a) totals[1 + a] += rho[s] * u[a * V + s];
                }
        }
    }
    free(fs); free(F); free(rho); free(u);
    return 0;
}

int SYM(real_size)(void) { return (int)sizeof(real); }

/* Threads the site loops run on (OpenMP), for reporting. */
int SYM(num_threads)(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
