/*
 * FP64 CPU oracle for the self-propelled DPD dimer model of Hinz, Panchenko,
 * Kim & Fried, "Particle-based simulations of self-motile suspensions"
 * (arXiv:1310.0998).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg and reference arm of the benchmark may load
 * it.  It shares no
 * code, header, constant table or helper with the CUDA library; the two are
 * written independently from the paper and from the published definition of
 * the Philox4x32-10 generator (Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).
 *
 * Bead i (0 <= i < n) is stored at index i ("id order").  Beads 2k and 2k+1
 * form dimer (agent) k; bead 2k is the head.
 *
 * What each function follows:
 *   orc_philox4x32_10   Philox4x32-10, SC'11 paper (round function, Weyl key
 *                       schedule, 10 rounds).
 *   orc_alpha           the random number alpha^ij of Sec. 2.1, Eq. (DPDcdr)_3:
 *                       zero mean, unit variance, symmetric in (i, j).
 *   orc_forces          Sec. 2, Eqs. (DPDf), (DPDcdr), (weightFunc01),
 *                       (stiffSpring), (DPDnp) and the director n^k; all-pairs
 *                       O(N^2) search with the minimum-image convention of the
 *                       periodic square domain of Sec. 5.
 *   orc_run             Newton's equations (Newton) advanced by the standard
 *                       velocity-Verlet scheme named in Sec. 5.
 *   orc_forces_cells    the same forces as orc_forces through a cell list
 *                       (OpenMP, one-sided, full 3x3 stencil); used to time a
 *                       CPU baseline and checked against orc_forces.
 *   orc_cell_counts     the cell-binning rule that the GPU path documents,
 *                       floor(x n_c / L) on the fixed-point position grid.
 *   orc_pair_counts     brute-force per-bead interacting-neighbour counts.
 *   orc3_forces,        the same force laws and velocity-Verlet in a periodic
 *   orc3_run            cube (three-dimensional variant), all pairs.
 *
 * Parity pins (tests/test_oracle_*.py): Philox against Triton's independent
 * Philox4x32-10 and against uniformity statistics; pair force against
 * hand-computed two- and three-bead cases; momentum conservation with drag and
 * propulsion off; the discrete momentum balance with them on; the single-dimer
 * drift recurrence and its limit f_p/zeta; the bond oscillation frequency;
 * the equilibrium temperature kBT; the cell-list variant against all pairs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Model parameters (Sec. 2 and Sec. 3; mass m of Eq. (Newton)). */
typedef struct {
    double L;       /* side of the periodic square domain                  */
    double a;       /* conservative amplitude A (Phi in Eq. (DPDcdrND2))   */
    double gamma;   /* pairwise friction gamma                             */
    double kBT;     /* reference energy k_B T                              */
    double rc;      /* cutoff radius r_c                                   */
    double kbond;   /* spring stiffness kappa, Eq. (stiffSpring)           */
    double r0;      /* spring rest length l, Eq. (stiffSpring)             */
    double fp;      /* self-propulsion magnitude f_SP, per bead            */
    double zeta;    /* Stokes friction gamma_s, Eq. (DPDnp)                */
    double dt;      /* time step Delta t                                   */
    double mass;    /* bead mass m                                         */
    uint64_t seed;  /* random-stream seed                                  */
    uint32_t replica;        /* replica number (XORed into the key)        */
    int32_t exclude_bonded;  /* 1: no pair force between bonded beads      */
    int32_t noise;           /* 0: uniform alpha, 1: Gaussian alpha        */
    int32_t pad;
    double wexp;             /* exponent s of the dissipative weight        */
                             /* w_D = w^s, w_R = w^(s/2); 0 selects s = 2   */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): 10 rounds of a 4-word bijection keyed by 2 words.  */
/* Round: (c0, c1, c2, c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2),                    */
/*                             hi(M0*c0)^c3^k1, lo(M0*c0)),                   */
/* with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped    */
/* by the Weyl constants (0x9E3779B9, 0xBB67AE85).                            */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Batch form for tests: n counters (4 words each) under one key. */
void orc_philox_batch(int64_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out)
{
    uint32_t key[2] = {k0, k1};
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* alpha^ij for the unordered bead pair {i, j} at force-evaluation step s.
 * Counter (min id, max id, s lo, s hi); key (seed lo, seed hi ^ replica).
 * Uniform variant: s24 = (2*(w0>>8) + 1 - 2^24) * 2^-24, an odd multiple of
 * 2^-24 in (-1, 1), symmetric about 0; alpha = sqrt(3) * s24 has zero mean and
 * unit variance.  Gaussian variant: Box-Muller on the top 24 bits of w0, w1. */
double orc_alpha(uint32_t i, uint32_t j, int64_t step, uint64_t seed, uint32_t replica, int noise)
{
    uint32_t lo = i < j ? i : j, hi = i < j ? j : i;
    uint32_t ctr[4] = {lo, hi, (uint32_t)((uint64_t)step & 0xffffffffu), (uint32_t)((uint64_t)step >> 32)};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ replica};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    if (noise == 0) {
        int32_t odd = (int32_t)(2u * (w[0] >> 8) + 1u) - (int32_t)(1 << 24);
        return sqrt(3.0) * ((double)odd * ldexp(1.0, -24));
    } else {
        double u1 = ((double)(w[0] >> 8) + 0.5) * ldexp(1.0, -24);
        double u2 = ((double)(w[1] >> 8) + 0.5) * ldexp(1.0, -24);
        return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    }
}

/* Minimum-image displacement in the periodic square of side L (Sec. 5). */
static double minimg(double d, double L)
{
    return d - L * nearbyint(d / L);
}

/* One DPD pair term, Eqs. (DPDf), (DPDcdr), (weightFunc01).  e = (r_i - r_j)/r,
 * so the conservative part A w e pushes i away from j (soft repulsion, Sec. 4).
 * The dissipative and random parts carry w_D = w^s and w_R = w^(s/2): s = 2 is
 * Eq. (DPDcdr) as printed; another s is the changed exponent of w that the
 * closing section proposes, with w_D = w_R^2 so that sigma^2 = 2 gamma kBT
 * still holds the temperature.
 * Returns 1 and the force on i when r < r_c and r > 0, else 0. */
static int pair_force(const orc_params *p, double dx, double dy, double dvx, double dvy,
                      uint32_t i, uint32_t j, int64_t step, double *fx, double *fy)
{
    double r2 = dx * dx + dy * dy;
    if (!(r2 < p->rc * p->rc) || r2 == 0.0) return 0;
    double r = sqrt(r2);
    double w = 1.0 - r / p->rc;
    double ex = dx / r, ey = dy / r;
    double dve = dvx * ex + dvy * ey;
    double sigma = sqrt(2.0 * p->gamma * p->kBT);
    double alpha = orc_alpha(i, j, step, p->seed, p->replica, p->noise);
    double s = p->wexp > 0.0 ? p->wexp : 2.0;
    double wd = s == 2.0 ? w * w : pow(w, s);
    double wr = s == 2.0 ? w : pow(w, 0.5 * s);
    double fc = p->a * w;
    double fd = -p->gamma * wd * dve;
    double fr = sigma * wr * alpha / sqrt(p->dt);
    double F = fc + fd + fr;
    *fx = F * ex;
    *fy = F * ey;
    return 1;
}

/* Non-pairwise and bond terms: harmonic bond, Eq. (stiffSpring), between beads
 * 2k and 2k+1; propulsion f_SP n^k on each bead of agent k with
 * n^k = (r_2k - r_2k+1)/|r_2k - r_2k+1|, Eq. (DPDnp); Stokes drag -gamma_s v on
 * every bead, Eq. (DPDnp). */
static void bonded_and_external(const orc_params *p, int64_t n, const double *x, const double *v, double *f)
{
    for (int64_t k = 0; k < n / 2; ++k) {
        int64_t i = 2 * k, j = 2 * k + 1;
        double dx = minimg(x[2 * i] - x[2 * j], p->L);
        double dy = minimg(x[2 * i + 1] - x[2 * j + 1], p->L);
        double r = sqrt(dx * dx + dy * dy);
        if (r > 0.0) {
            double nx = dx / r, ny = dy / r;
            double fb = -p->kbond * (r - p->r0);  /* -dV_H/dr along n, on i */
            f[2 * i] += fb * nx + p->fp * nx;
            f[2 * i + 1] += fb * ny + p->fp * ny;
            f[2 * j] += -fb * nx + p->fp * nx;
            f[2 * j + 1] += -fb * ny + p->fp * ny;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        f[2 * i] -= p->zeta * v[2 * i];
        f[2 * i + 1] -= p->zeta * v[2 * i + 1];
    }
}

/* Total force on every bead at positions x and velocities v, with the random
 * stream of force-evaluation step `step`.  x, v, f: [n][2] doubles.
 * Returns the number of interacting (r < r_c, non-excluded) pairs. */
int64_t orc_forces(const orc_params *p, int64_t n, const double *x, const double *v, int64_t step, double *f)
{
    int64_t npairs = 0;
    memset(f, 0, sizeof(double) * 2 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            if (p->exclude_bonded && (i ^ 1) == j) continue;
            double dx = minimg(x[2 * i] - x[2 * j], p->L);
            double dy = minimg(x[2 * i + 1] - x[2 * j + 1], p->L);
            double fx, fy;
            if (pair_force(p, dx, dy, v[2 * i] - v[2 * j], v[2 * i + 1] - v[2 * j + 1],
                           (uint32_t)i, (uint32_t)j, step, &fx, &fy)) {
                f[2 * i] += fx; f[2 * i + 1] += fy;
                f[2 * j] -= fx; f[2 * j + 1] -= fy;
                ++npairs;
            }
        }
    }
    bonded_and_external(p, n, x, v, f);
    return npairs;
}

/* Only the pairwise part (for the hand-computed pins). */
void orc_pair_forces_only(const orc_params *p, int64_t n, const double *x, const double *v, int64_t step, double *f)
{
    memset(f, 0, sizeof(double) * 2 * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            if (p->exclude_bonded && (i ^ 1) == j) continue;
            double fx, fy;
            double dx = minimg(x[2 * i] - x[2 * j], p->L);
            double dy = minimg(x[2 * i + 1] - x[2 * j + 1], p->L);
            if (pair_force(p, dx, dy, v[2 * i] - v[2 * j], v[2 * i + 1] - v[2 * j + 1],
                           (uint32_t)i, (uint32_t)j, step, &fx, &fy)) {
                f[2 * i] += fx; f[2 * i + 1] += fy;
                f[2 * j] -= fx; f[2 * j + 1] -= fy;
            }
        }
}

static void wrap_positions(const orc_params *p, int64_t n, double *x)
{
    for (int64_t k = 0; k < 2 * n; ++k) x[k] -= p->L * floor(x[k] / p->L);
}

/* Cell-list force evaluation (OpenMP).  Cells of side >= r_c on an nc x nc
 * grid; every bead visits the 3x3 block of cells around its own and keeps only
 * its own side of each pair (no Newton-3), so each pair's random number is
 * drawn twice, identically.  Same arithmetic per pair as orc_forces.  Requires
 * nc >= 3.  Returns the number of interacting pairs. */
int64_t orc_forces_cells(const orc_params *p, int64_t n, const double *x, const double *v, int64_t step, double *f)
{
    /* a hair of margin keeps cells strictly wider than r_c after rounding */
    int nc = (int)floor(p->L / (p->rc * (1.0 + 1e-9)));
    if (nc < 3) return orc_forces(p, n, x, v, step, f);
    double cs = p->L / nc;
    int64_t ncell = (int64_t)nc * nc;
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memset(head, 0, sizeof(int64_t) * (size_t)(ncell + 1));
    for (int64_t i = 0; i < n; ++i) {
        int cx = (int)floor(x[2 * i] / cs), cy = (int)floor(x[2 * i + 1] / cs);
        cx = cx < 0 ? 0 : (cx >= nc ? nc - 1 : cx);
        cy = cy < 0 ? 0 : (cy >= nc ? nc - 1 : cy);
        cell[i] = (int64_t)cy * nc + cx;
        head[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) head[c + 1] += head[c];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
        memcpy(fill, head, sizeof(int64_t) * (size_t)ncell);
        for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = i;
        free(fill);
    }
    int64_t npairs2 = 0;
#pragma omp parallel for schedule(static) reduction(+ : npairs2)
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0;
        int cx = (int)(cell[i] % nc), cy = (int)(cell[i] / nc);
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int nx = (cx + ox + nc) % nc, ny = (cy + oy + nc) % nc;
                int64_t c = (int64_t)ny * nc + nx;
                for (int64_t q = head[c]; q < head[c + 1]; ++q) {
                    int64_t j = order[q];
                    if (j == i) continue;
                    if (p->exclude_bonded && (i ^ 1) == j) continue;
                    double dx = minimg(x[2 * i] - x[2 * j], p->L);
                    double dy = minimg(x[2 * i + 1] - x[2 * j + 1], p->L);
                    double gx, gy;
                    if (pair_force(p, dx, dy, v[2 * i] - v[2 * j], v[2 * i + 1] - v[2 * j + 1],
                                   (uint32_t)i, (uint32_t)j, step, &gx, &gy)) {
                        fx += gx; fy += gy; ++npairs2;
                    }
                }
            }
        f[2 * i] = fx;
        f[2 * i + 1] = fy;
    }
    free(head); free(order); free(cell);
    bonded_and_external(p, n, x, v, f);
    return npairs2 / 2;
}

/* Standard velocity-Verlet, Sec. 5: per step s -> s+1
 *   v <- v + (dt/2m) f_s;  x <- wrap(x + dt v);  f_{s+1} = F(x, v, s+1);
 *   v <- v + (dt/2m) f_{s+1}.
 * The dissipative and drag terms see the half-step velocity.  On entry f holds
 * f_s at *step; on exit x, v, f are at *step + nsteps.  If thermo != NULL it
 * receives per step (KE, Px, Py, Fx_sum, Fy_sum) after each full step.
 * use_cells selects orc_forces_cells. */
void orc_run(const orc_params *p, int64_t n, double *x, double *v, double *f, int64_t *step,
             int64_t nsteps, int use_cells, double *thermo)
{
    double h = 0.5 * p->dt / p->mass;
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int64_t k = 0; k < 2 * n; ++k) v[k] += h * f[k];
        for (int64_t k = 0; k < 2 * n; ++k) x[k] += p->dt * v[k];
        wrap_positions(p, n, x);
        *step += 1;
        if (use_cells) orc_forces_cells(p, n, x, v, *step, f);
        else orc_forces(p, n, x, v, *step, f);
        for (int64_t k = 0; k < 2 * n; ++k) v[k] += h * f[k];
        if (thermo) {
            double ke = 0, px = 0, py = 0, fx = 0, fy = 0;
            for (int64_t i = 0; i < n; ++i) {
                ke += 0.5 * p->mass * (v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1]);
                px += p->mass * v[2 * i];
                py += p->mass * v[2 * i + 1];
                fx += f[2 * i];
                fy += f[2 * i + 1];
            }
            thermo[5 * s + 0] = ke; thermo[5 * s + 1] = px; thermo[5 * s + 2] = py;
            thermo[5 * s + 3] = fx; thermo[5 * s + 4] = fy;
        }
    }
}

/* Cell binning, the rule the GPU path documents: with n_c cells per side,
 * bead x lies in cell floor(x n_c / L).  Positions are on the grid
 * x = X L / 2^32 (integer X), so X = x / L * 2^32 exactly and the cell is
 * (X n_c) >> 32 in integer arithmetic.  counts: [nc*nc], row-major. */
void orc_cell_counts(int64_t n, const double *x, double L, int32_t nc, uint32_t *counts)
{
    memset(counts, 0, sizeof(uint32_t) * (size_t)nc * (size_t)nc);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t X = (uint64_t)(x[2 * i] / L * 4294967296.0);
        uint64_t Y = (uint64_t)(x[2 * i + 1] / L * 4294967296.0);
        uint64_t cx = (X * (uint64_t)nc) >> 32, cy = (Y * (uint64_t)nc) >> 32;
        counts[cy * (uint64_t)nc + cx]++;
    }
}

/* Brute-force per-bead interacting-neighbour counts in FP64 on the given
 * positions: pairs with r < r_c, r > 0, excluding the bonded partner when
 * exclude_bonded.  A pair with |r^2 - r_c^2| < tie * r_c^2 is "ambiguous": it
 * is not counted in cnt but in amb (per bead).  Returns the unambiguous pair
 * total. */
int64_t orc_pair_counts(const orc_params *p, int64_t n, const double *x, double tie, uint32_t *cnt, uint32_t *amb)
{
    int64_t total = 0;
    double rc2 = p->rc * p->rc;
    memset(cnt, 0, sizeof(uint32_t) * (size_t)n);
    memset(amb, 0, sizeof(uint32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            if (p->exclude_bonded && (i ^ 1) == j) continue;
            double dx = minimg(x[2 * i] - x[2 * j], p->L);
            double dy = minimg(x[2 * i + 1] - x[2 * j + 1], p->L);
            double r2 = dx * dx + dy * dy;
            if (fabs(r2 - rc2) < tie * rc2) { amb[i]++; amb[j]++; continue; }
            if (r2 < rc2 && r2 > 0.0) { cnt[i]++; cnt[j]++; ++total; }
        }
    return total;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Three-dimensional variant.  Sec. 2 writes every force as a vector law, so  */
/* the same Eqs. (DPDf), (DPDcdr), (weightFunc01), (stiffSpring), (DPDnp)     */
/* apply unchanged in a periodic cube of side L; x, v, f: [n][3] doubles.     */
/* ------------------------------------------------------------------------ */
static int pair_force3(const orc_params *p, const double d[3], const double dv[3], uint32_t i, uint32_t j,
                       int64_t step, double F3[3])
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < p->rc * p->rc) || r2 == 0.0) return 0;
    double r = sqrt(r2);
    double w = 1.0 - r / p->rc;
    double e[3] = {d[0] / r, d[1] / r, d[2] / r};
    double dve = dv[0] * e[0] + dv[1] * e[1] + dv[2] * e[2];
    double sigma = sqrt(2.0 * p->gamma * p->kBT);
    double alpha = orc_alpha(i, j, step, p->seed, p->replica, p->noise);
    double s = p->wexp > 0.0 ? p->wexp : 2.0;
    double wd = s == 2.0 ? w * w : pow(w, s);
    double wr = s == 2.0 ? w : pow(w, 0.5 * s);
    double F = p->a * w - p->gamma * wd * dve + sigma * wr * alpha / sqrt(p->dt);
    for (int c = 0; c < 3; ++c) F3[c] = F * e[c];
    return 1;
}

static void bonded_and_external3(const orc_params *p, int64_t n, const double *x, const double *v, double *f)
{
    for (int64_t k = 0; k < n / 2; ++k) {
        int64_t i = 2 * k, j = 2 * k + 1;
        double d[3], r2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            d[c] = minimg(x[3 * i + c] - x[3 * j + c], p->L);
            r2 += d[c] * d[c];
        }
        double r = sqrt(r2);
        if (r > 0.0) {
            double fb = -p->kbond * (r - p->r0);
            for (int c = 0; c < 3; ++c) {
                double nc = d[c] / r;
                f[3 * i + c] += fb * nc + p->fp * nc;
                f[3 * j + c] += -fb * nc + p->fp * nc;
            }
        }
    }
    for (int64_t k = 0; k < 3 * n; ++k) f[k] -= p->zeta * v[k];
}

int64_t orc3_forces(const orc_params *p, int64_t n, const double *x, const double *v, int64_t step, double *f)
{
    int64_t npairs = 0;
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            if (p->exclude_bonded && (i ^ 1) == j) continue;
            double d[3], dv[3], F3[3];
            for (int c = 0; c < 3; ++c) {
                d[c] = minimg(x[3 * i + c] - x[3 * j + c], p->L);
                dv[c] = v[3 * i + c] - v[3 * j + c];
            }
            if (pair_force3(p, d, dv, (uint32_t)i, (uint32_t)j, step, F3)) {
                for (int c = 0; c < 3; ++c) {
                    f[3 * i + c] += F3[c];
                    f[3 * j + c] -= F3[c];
                }
                ++npairs;
            }
        }
    bonded_and_external3(p, n, x, v, f);
    return npairs;
}

/* Velocity-Verlet in the cube, as orc_run; thermo per step: (KE, Px, Py, Pz,
 * 0). */
void orc3_run(const orc_params *p, int64_t n, double *x, double *v, double *f, int64_t *step, int64_t nsteps,
              double *thermo)
{
    double h = 0.5 * p->dt / p->mass;
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int64_t k = 0; k < 3 * n; ++k) v[k] += h * f[k];
        for (int64_t k = 0; k < 3 * n; ++k) {
            x[k] += p->dt * v[k];
            x[k] -= p->L * floor(x[k] / p->L);
        }
        *step += 1;
        orc3_forces(p, n, x, v, *step, f);
        for (int64_t k = 0; k < 3 * n; ++k) v[k] += h * f[k];
        if (thermo) {
            double ke = 0, P[3] = {0, 0, 0};
            for (int64_t i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) {
                    ke += 0.5 * p->mass * v[3 * i + c] * v[3 * i + c];
                    P[c] += p->mass * v[3 * i + c];
                }
            thermo[5 * s + 0] = ke; thermo[5 * s + 1] = P[0]; thermo[5 * s + 2] = P[1];
            thermo[5 * s + 3] = P[2]; thermo[5 * s + 4] = 0.0;
        }
    }
}
