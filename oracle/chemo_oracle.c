/*
 * chemo_oracle.c -- plain FP64 CPU oracle for one time step of the hybrid
 * chemotaxis model of Bruna, Maini & Robinson, "Particle-based simulations of
 * reaction-diffusion processes with Aboria" (arXiv:1805.11007).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * CPU-baseline / reference legs of the benchmark load this library. The GPU
 * library never links, calls or includes anything from this directory, and
 * this file includes nothing from the GPU library.
 *
 * Every function is a slow, direct restatement of one piece of the paper's
 * method in double precision, applied in the order the paper applies it
 * (Sect. 3: gradient of c, interpolation to the cells, pair interaction,
 * Euler-Maruyama move, boundary handling, density estimate on the grid, PDE
 * update). Where the paper is silent or inconsistent, the reading taken is
 * stated next to the code that implements it.
 *
 * Parity pins: every exported function is pinned by tests that do not use
 * this file's own formulas (brute-force pair search, closed forms, discrete
 * conservation laws, eigenmodes, library Philox); see the test suite.
 *
 * Layouts: positions are n x dim row-major doubles; grids are C-order
 * [z][y][x] with x fastest (2D: [y][x]).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_SPECIES 8

/* Model parameters, as the oracle reads them (its own definition). */
#define ORC_PI 3.14159265358979323846

typedef struct orc_params {
    int32_t dim;          /* 2 or 3 (the paper works in 2D, Sect. 2) */
    int32_t boundary;     /* 0 reflecting walls (Sect. 3.2), 1 periodic (Sect. 4) */
    double lo[3], hi[3];  /* domain box */
    int32_t n_species;
    double diameter[ORC_MAX_SPECIES];    /* sigma_s: epsilon_ij = (sigma_i+sigma_j)/2 */
    double D[ORC_MAX_SPECIES];           /* diffusivity per species, Eq. (1a)/(1b) */
    double chemotactic[ORC_MAX_SPECIES]; /* multiplier of chi, Eq. (1b): beta=1, alpha=0 */
    double secrete[ORC_MAX_SPECIES];     /* k_s, source term of Eq. (1d) */
    double consume[ORC_MAX_SPECIES];     /* kappa_s, consumption term of Eq. (1d) */
    double react_k0[ORC_MAX_SPECIES];    /* constant switching rate, Eq. (1c) */
    double react_kc[ORC_MAX_SPECIES];    /* switching rate per unit c, Eq. (1c) */
    int32_t react_to[ORC_MAX_SPECIES];   /* species a cell switches to */
    int32_t reactions;                   /* 0 off, 1 fixed-step reactions (Sect. 2.1) */
    double chi;                          /* chemotactic sensitivity, Eq. (1b) */
    double inter;                        /* interaction strength of the Sect. 3.2 force */
    double cutoff_factor;                /* r_c,ij = cutoff_factor * epsilon_ij */
    int32_t cutoff_mode;                 /* 0 hard truncation, 1 force shifted to 0 at r_c */
    int32_t chem_mode;                   /* 0 grid PDE, 1 fixed gradient (Sect. 4, c = x) */
    double fixed_grad[3];
    int32_t grid[3];                     /* nodes per axis */
    double Dc, gamma;                    /* chemical diffusivity and decay, Eq. (1d) */
    int32_t pde_bc;                      /* 0 Neumann (no flux), 1 Dirichlet (held), 2 periodic */
    int32_t pde_substeps;                /* 0 = automatic (see orc_substeps) */
    double dt;
    uint64_t seed;
    int32_t move_scheme;   /* 0 Euler-Maruyama (Eq. (2)), 1 tamed Euler (Sect. 3.2, Eq. sde_ETamed) */
    int32_t hard_sphere;   /* 1: overlap correction after the move (Sect. 3.2, hard spheres) */
    int32_t deposit_kernel;/* 0 cloud-in-cell (Sect. 2.3), 1 Gaussian kernel density estimate (Sect. 2.3) */
    double kde_range;      /* KDE truncation radius in bandwidths (bandwidth = cell diameter) */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Threads                                                                   */
/* ------------------------------------------------------------------------ */

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 Philox S-box with a Weyl  */
/* key schedule. Written from that definition.                               */
/* ------------------------------------------------------------------------ */

#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Batched form for tests: ctr is n x 4, out is n x 4. */
void orc_philox_batch(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Stream tags of the counter (third word). */
#define ORC_TAG_MOVE 0u
#define ORC_TAG_REACT 2u

/* The four Philox words of cell `id` at step `step` on stream `tag`:
 * key = (seed lo, seed hi), counter = (id, step lo, tag, step hi). */
static void orc_words(uint64_t seed, uint32_t id, uint64_t step, uint32_t tag, uint32_t w[4])
{
    uint32_t ctr[4] = {id, (uint32_t)step, tag, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

/* A 32-bit word as a uniform on (0,1): u = (w + 1/2) 2^-32 (exact in FP64). */
static double orc_uniform(uint32_t w)
{
    return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

/* Four standard normals by the Box-Muller transform of the two uniform pairs
 * (u0,u1) and (u2,u3); these are the xi_i of Eq. (2). */
void orc_normals(uint64_t seed, uint32_t id, uint64_t step, uint32_t tag, double xi[4])
{
    uint32_t w[4];
    orc_words(seed, id, step, tag, w);
    const double two_pi = 6.283185307179586476925286766559;
    double u0 = orc_uniform(w[0]), u1 = orc_uniform(w[1]);
    double u2 = orc_uniform(w[2]), u3 = orc_uniform(w[3]);
    double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    xi[0] = r0 * cos(two_pi * u1);
    xi[1] = r0 * sin(two_pi * u1);
    xi[2] = r1 * cos(two_pi * u3);
    xi[3] = r1 * sin(two_pi * u3);
}

void orc_normals_batch(uint64_t seed, int64_t n, const uint32_t *ids, uint64_t step,
                       uint32_t tag, double *xi)
{
    for (int64_t i = 0; i < n; ++i) orc_normals(seed, ids[i], step, tag, xi + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers                                                          */
/* ------------------------------------------------------------------------ */

static double orc_len(const orc_params *p, int a) { return p->hi[a] - p->lo[a]; }

/* Minimum-image displacement along axis a under periodicity (Sect. 3.2: the
 * search returns the shortest vector between two particles). */
static double orc_wrap_delta(const orc_params *p, int a, double d)
{
    if (p->boundary == 1) {
        double L = orc_len(p, a);
        d -= L * floor(d / L + 0.5);
    }
    return d;
}

/* ------------------------------------------------------------------------ */
/* Cell-list bin of each particle with the FP32 rule of the GPU library:     */
/*   nb = max(1, floor(L / b)), inv_b = (float)(nb / L),                     */
/*   cell = clamp((int)floorf(((float)x - (float)lo) * inv_b), 0, nb - 1).   */
/* Evaluated here in single precision so that bins can be compared exactly.  */
/* ------------------------------------------------------------------------ */

void orc_bins_f32(const orc_params *p, double bin_side, int64_t n, const float *pos,
                  int32_t *cells, int32_t nb_out[3])
{
    int32_t nb[3] = {1, 1, 1};
    float inv_b[3] = {0.f, 0.f, 0.f}, lo_f[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < p->dim; ++a) {
        double L = orc_len(p, a);
        double m = floor(L / bin_side);
        nb[a] = m < 1.0 ? 1 : (int32_t)m;
        inv_b[a] = (float)((double)nb[a] / L);
        lo_f[a] = (float)p->lo[a];
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < p->dim; ++a) {
            volatile float rel = pos[i * p->dim + a] - lo_f[a];
            volatile float t = rel * inv_b[a];
            int c = (int)floorf(t);
            if (c < 0) c = 0;
            if (c > nb[a] - 1) c = nb[a] - 1;
            cells[i * p->dim + a] = c;
        }
    }
    for (int a = 0; a < 3; ++a) nb_out[a] = nb[a];
}

/* ------------------------------------------------------------------------ */
/* Pair interaction (Sect. 3.2 interaction loop; Eq. (1a)/(1b) pair term).  */
/* u(r) = exp(-r/eps) (Sect. 3), so -grad_i u = (1/eps) e^{-r/eps} (X_i-X_j)/r, */
/* scaled by `inter`. Heterogeneous sizes: eps_ij = (sigma_i+sigma_j)/2, the  */
/* contact distance used for hard spheres in Sect. 2.2. The search radius is */
/* r_c,ij = cutoff_factor * eps_ij; coincident particles (r = 0) get no force */
/* (the paper tests r > 0).                                                  */
/* ------------------------------------------------------------------------ */

typedef struct orc_pair_geom {
    double d[3];   /* X_i - X_j, minimum image */
    double r2, r, eps, rc;
} orc_pair_geom;

static void orc_geom(const orc_params *p, const double *xi, const double *xj, int si, int sj,
                     orc_pair_geom *g)
{
    g->r2 = 0.0;
    for (int a = 0; a < p->dim; ++a) {
        g->d[a] = orc_wrap_delta(p, a, xi[a] - xj[a]);
        g->r2 += g->d[a] * g->d[a];
    }
    g->r = sqrt(g->r2);
    g->eps = 0.5 * (p->diameter[si] + p->diameter[sj]);
    g->rc = p->cutoff_factor * g->eps;
}

/* Magnitude of the pair force at distance r (r inside the cutoff). */
static double orc_force_mag(const orc_params *p, double r, double eps)
{
    double f = exp(-r / eps);
    if (p->cutoff_mode == 1) f -= exp(-p->cutoff_factor);
    return p->inter / eps * f;
}

/* Borderline pairs: |r^2 - r_c^2| <= 1e-6 r_c^2; an FP32 evaluation may
 * classify these either way. */
static int orc_is_border(const orc_pair_geom *g)
{
    return fabs(g->r2 - g->rc * g->rc) <= 1e-6 * g->rc * g->rc;
}

static double orc_max_cutoff(const orc_params *p)
{
    double m = 0.0;
    for (int s = 0; s < p->n_species; ++s)
        for (int t = 0; t < p->n_species; ++t) {
            double eps = 0.5 * (p->diameter[s] + p->diameter[t]);
            double rc = p->cutoff_factor * eps;
            if (rc > m) m = rc;
            if (p->hard_sphere && eps > m) m = eps;  /* contact distance of the correction */
        }
    return m;
}

/* The oracle's own cell list: cells of side >= max cutoff, a linked list per
 * cell, and a search over the 3^d surrounding cells. Falls back to all pairs
 * when an axis has fewer than 3 cells (so no cell is visited twice). */
typedef struct orc_cells {
    int nc[3];
    double side[3];
    int64_t ncell;
    int64_t *head, *next;
    int brute;
} orc_cells;

static void orc_cells_build(const orc_params *p, int64_t n, const double *pos, orc_cells *cl)
{
    double rcmax = orc_max_cutoff(p);
    cl->brute = 0;
    cl->ncell = 1;
    for (int a = 0; a < 3; ++a) { cl->nc[a] = 1; cl->side[a] = 1.0; }
    for (int a = 0; a < p->dim; ++a) {
        double L = orc_len(p, a);
        int m = rcmax > 0.0 ? (int)floor(L / rcmax) : 1;
        if (m > 1024) m = 1024;
        if (m < 3) cl->brute = 1;
        if (m < 1) m = 1;
        cl->nc[a] = m;
        cl->side[a] = L / m;
        cl->ncell *= m;
    }
    cl->head = NULL;
    cl->next = NULL;
    if (cl->brute) return;
    cl->head = (int64_t *)malloc(sizeof(int64_t) * (size_t)cl->ncell);
    cl->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < cl->ncell; ++c) cl->head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t lin = 0, stride = 1;
        for (int a = 0; a < p->dim; ++a) {
            int c = (int)floor((pos[i * p->dim + a] - p->lo[a]) / cl->side[a]);
            if (c < 0) c = 0;
            if (c >= cl->nc[a]) c = cl->nc[a] - 1;
            lin += c * stride;
            stride *= cl->nc[a];
        }
        cl->next[i] = cl->head[lin];
        cl->head[lin] = i;
    }
}

static void orc_cells_free(orc_cells *cl)
{
    free(cl->head);
    free(cl->next);
}

/* Calls visit(j) for every candidate j of particle i (a superset of the
 * particles within the maximum cutoff), each candidate once. */
typedef void (*orc_visit_fn)(void *ctx, int64_t j);

static void orc_candidates(const orc_params *p, const orc_cells *cl, int64_t n, const double *pos,
                           int64_t i, orc_visit_fn visit, void *ctx)
{
    if (cl->brute) {
        for (int64_t j = 0; j < n; ++j) visit(ctx, j);
        return;
    }
    int ci[3] = {0, 0, 0};
    for (int a = 0; a < p->dim; ++a) {
        int c = (int)floor((pos[i * p->dim + a] - p->lo[a]) / cl->side[a]);
        if (c < 0) c = 0;
        if (c >= cl->nc[a]) c = cl->nc[a] - 1;
        ci[a] = c;
    }
    int zlo = p->dim == 3 ? -1 : 0, zhi = p->dim == 3 ? 1 : 0;
    for (int oz = zlo; oz <= zhi; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int off[3] = {ox, oy, oz};
                int64_t lin = 0, stride = 1;
                int skip = 0;
                for (int a = 0; a < p->dim; ++a) {
                    int c = ci[a] + off[a];
                    if (c < 0 || c >= cl->nc[a]) {
                        if (p->boundary == 1)
                            c = (c + cl->nc[a]) % cl->nc[a];
                        else
                            skip = 1;
                    }
                    lin += c * stride;
                    stride *= cl->nc[a];
                }
                if (skip) continue;
                for (int64_t j = cl->head[lin]; j >= 0; j = cl->next[j]) visit(ctx, j);
            }
}

/* Per-particle accumulation of the pair force. */
typedef struct orc_force_ctx {
    const orc_params *p;
    const double *pos;
    const uint8_t *sp;
    int64_t i;
    double F[3];
    double fabs_sum;   /* sum_j |f_ij| over included pairs */
    double border;     /* sum_j |f_ij| over borderline pairs (included or not) */
    int64_t count;     /* number of included neighbours */
    uint64_t idsum;    /* sum of included neighbour indices */
    uint64_t idxor;    /* xor of included neighbour indices */
} orc_force_ctx;

static void orc_force_visit(void *vctx, int64_t j)
{
    orc_force_ctx *c = (orc_force_ctx *)vctx;
    if (j == c->i) return;
    const orc_params *p = c->p;
    orc_pair_geom g;
    orc_geom(p, c->pos + c->i * p->dim, c->pos + j * p->dim, c->sp[c->i], c->sp[j], &g);
    int border = orc_is_border(&g);
    if (border) {
        double rb = g.r > 0.0 ? g.r : g.rc;
        double f = p->inter / g.eps * exp(-rb / g.eps);
        c->border += fabs(f);
    }
    if (!(g.r > 0.0) || !(g.r < g.rc)) return;
    double f = orc_force_mag(p, g.r, g.eps);
    for (int a = 0; a < p->dim; ++a) c->F[a] += f * g.d[a] / g.r;
    c->fabs_sum += fabs(f);
    c->count += 1;
    c->idsum += (uint64_t)j;
    c->idxor ^= (uint64_t)j;
}

/* Pair force F_i = sum_{j != i, 0 < r < r_c} f(r) (X_i - X_j)/r for every
 * particle. method 0: all pairs; 1: the oracle's cell list. Optional outputs
 * (NULL to skip): fabs_sum[n], border[n], count[n], idsum[n], idxor[n]. */
void orc_pair_forces(const orc_params *p, int64_t n, const double *pos, const uint8_t *sp,
                     int method, double *F, double *fabs_sum, double *border, int64_t *count,
                     uint64_t *idsum, uint64_t *idxor)
{
    orc_cells cl;
    memset(&cl, 0, sizeof(cl));
    if (method == 1)
        orc_cells_build(p, n, pos, &cl);
    else
        cl.brute = 1;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        orc_force_ctx c;
        memset(&c, 0, sizeof(c));
        c.p = p;
        c.pos = pos;
        c.sp = sp;
        c.i = i;
        orc_candidates(p, &cl, n, pos, i, orc_force_visit, &c);
        for (int a = 0; a < p->dim; ++a) F[i * p->dim + a] = c.F[a];
        if (fabs_sum) fabs_sum[i] = c.fabs_sum;
        if (border) border[i] = c.border;
        if (count) count[i] = c.count;
        if (idsum) idsum[i] = c.idsum;
        if (idxor) idxor[i] = c.idxor;
    }
    orc_cells_free(&cl);
}

/* ------------------------------------------------------------------------ */
/* Chemical grid (Sect. 3.5). Node k sits at lo + k h. Non-periodic grids    */
/* include both walls, h = L/(N-1); periodic grids omit the duplicate node,  */
/* h = L/N. (The paper places p_0 at min with spacing hc; its interpolation  */
/* multiplies by Nc where 1/hc is meant.)                                    */
/* ------------------------------------------------------------------------ */

static int orc_gdim(const orc_params *p, int a) { return a < p->dim ? p->grid[a] : 1; }

double orc_grid_h(const orc_params *p, int a)
{
    int N = p->grid[a];
    double L = orc_len(p, a);
    return p->pde_bc == 2 ? L / N : L / (N - 1);
}

int64_t orc_grid_size(const orc_params *p)
{
    int64_t G = 1;
    for (int a = 0; a < p->dim; ++a) G *= p->grid[a];
    return G;
}

static int64_t orc_gidx(const orc_params *p, const int k[3])
{
    return (int64_t)k[0] + (int64_t)orc_gdim(p, 0) * ((int64_t)k[1] + (int64_t)orc_gdim(p, 1) * k[2]);
}

/* Neighbour node index along an axis with the ghost rule of the boundary:
 * Neumann / Dirichlet mirror (c_{-1} = c_1, c_N = c_{N-2}); periodic wraps. */
static int orc_nbr(const orc_params *p, int a, int k)
{
    int N = p->grid[a];
    if (p->pde_bc == 2) return (k % N + N) % N;
    if (k < 0) return -k;
    if (k > N - 1) return 2 * (N - 1) - k;
    return k;
}

/* Number of PDE substeps per particle step. The explicit scheme of Sect. 3.5
 * (centred differences, forward Euler) is stable only for
 * 2 d D_c dt_s / h^2 <= 1; the step is split into
 * s = ceil((sum_a 2 D_c dt / h_a^2) / 0.9) equal substeps (at least 1). */
int orc_substeps(const orc_params *p)
{
    if (p->pde_substeps > 0) return p->pde_substeps;
    double lam = 0.0;
    for (int a = 0; a < p->dim; ++a) {
        double h = orc_grid_h(p, a);
        lam += 2.0 * p->Dc * p->dt / (h * h);
    }
    int s = (int)ceil(lam / 0.9);
    return s < 1 ? 1 : s;
}

/* Cell of the grid containing x along axis a and the fractional offset in it
 * (linear interpolation, Sect. 2.3 / 3.6). Non-periodic: the cell index is
 * clamped to [0, N-2], so x = hi uses the last cell with offset 1. */
static void orc_cell_frac(const orc_params *p, int a, double x, int *k0, int *k1, double *f)
{
    int N = p->grid[a];
    double h = orc_grid_h(p, a);
    double t = (x - p->lo[a]) / h;
    if (p->pde_bc == 2) {
        double fl = floor(t);
        int k = (int)fl;
        *f = t - fl;
        k = ((k % N) + N) % N;
        *k0 = k;
        *k1 = (k + 1) % N;
    } else {
        int k = (int)floor(t);
        if (k < 0) k = 0;
        if (k > N - 2) k = N - 2;
        *f = t - k;
        *k0 = k;
        *k1 = k + 1;
    }
}

/* Central-difference gradient of c at node k (the D1x/D1y operators of
 * Sect. 3.5), component a. Wall nodes use the mirror ghost, which gives a zero
 * normal component (no flux). */
static double orc_node_grad(const orc_params *p, const double *c, const int k[3], int a)
{
    int kp[3] = {k[0], k[1], k[2]}, km[3] = {k[0], k[1], k[2]};
    kp[a] = orc_nbr(p, a, k[a] + 1);
    km[a] = orc_nbr(p, a, k[a] - 1);
    return (c[orc_gidx(p, kp)] - c[orc_gidx(p, km)]) / (2.0 * orc_grid_h(p, a));
}

/* Linear (bilinear in 2D, trilinear in 3D) interpolation weights of the 2^d
 * nodes around x. Returns the number of corners. */
static int orc_corners(const orc_params *p, const double *x, int nodes[8][3], double w[8])
{
    int k0[3] = {0, 0, 0}, k1[3] = {0, 0, 0};
    double f[3] = {0, 0, 0};
    for (int a = 0; a < p->dim; ++a) orc_cell_frac(p, a, x[a], &k0[a], &k1[a], &f[a]);
    int nc = 1 << p->dim;
    for (int m = 0; m < nc; ++m) {
        double wt = 1.0;
        for (int a = 0; a < 3; ++a) {
            int bit = (m >> a) & 1;
            if (a < p->dim) {
                nodes[m][a] = bit ? k1[a] : k0[a];
                wt *= bit ? f[a] : (1.0 - f[a]);
            } else {
                nodes[m][a] = 0;
            }
        }
        w[m] = wt;
    }
    return nc;
}

/* Chemotactic drift chi * chemotactic_s * grad c(X_i) for every particle
 * (Eq. (1b); Sect. 3.6). The gradient is the central difference at the grid
 * nodes, interpolated linearly in every axis to X_i (the paper interpolates
 * each component along its own axis only; the full multilinear form
 * reproduces the same linear fields). chem_mode 1 uses the fixed gradient. */
void orc_drift(const orc_params *p, int64_t n, const double *pos, const uint8_t *sp,
               const double *c, double *drift)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double g[3] = {0, 0, 0};
        double scale = p->chi * p->chemotactic[sp[i]];
        if (scale != 0.0) {
            if (p->chem_mode == 1) {
                for (int a = 0; a < p->dim; ++a) g[a] = p->fixed_grad[a];
            } else {
                int nodes[8][3];
                double w[8];
                int nc = orc_corners(p, pos + i * p->dim, nodes, w);
                for (int m = 0; m < nc; ++m)
                    for (int a = 0; a < p->dim; ++a) g[a] += w[m] * orc_node_grad(p, c, nodes[m], a);
            }
        }
        for (int a = 0; a < p->dim; ++a) drift[i * p->dim + a] = scale * g[a];
    }
}

/* Interpolated concentration c(X_i) (Sect. 3.6), used by the reaction rate. */
void orc_conc(const orc_params *p, int64_t n, const double *pos, const double *c, double *conc)
{
    for (int64_t i = 0; i < n; ++i) {
        int nodes[8][3];
        double w[8];
        double v = 0.0;
        if (p->chem_mode == 0) {
            int nc = orc_corners(p, pos + i * p->dim, nodes, w);
            for (int m = 0; m < nc; ++m) v += w[m] * c[orc_gidx(p, nodes[m])];
        } else {
            for (int a = 0; a < p->dim; ++a) v += p->fixed_grad[a] * (pos[i * p->dim + a] - p->lo[a]);
        }
        conc[i] = v;
    }
}

/* Trapezoid weight of a node: 1/2 per axis on which it lies on a wall. */
static double orc_tau(const orc_params *p, const int k[3])
{
    double t = 1.0;
    if (p->pde_bc == 2) return t;
    for (int a = 0; a < p->dim; ++a)
        if (k[a] == 0 || k[a] == p->grid[a] - 1) t *= 0.5;
    return t;
}

/* Cloud-in-cell density estimate of the random measures of Eq. (1e)
 * (particle-in-cell with linear weights, Sect. 2.3): each cell's unit mass is
 * split over the 2^d surrounding nodes with the interpolation weights, and a
 * node's density is its mass over its control volume tau_k h^d. Outputs the
 * per-step source S_k = dt sum_i k_{s_i} w_ik / (tau_k h^d) and the
 * consumption coefficient R_k = sum_i kappa_{s_i} w_ik / (tau_k h^d). */
void orc_deposit(const orc_params *p, int64_t n, const double *pos, const uint8_t *sp, double *S,
                 double *R)
{
    int64_t G = orc_grid_size(p);
    double hd = 1.0;
    for (int a = 0; a < p->dim; ++a) hd *= orc_grid_h(p, a);
    for (int64_t k = 0; k < G; ++k) {
        S[k] = 0.0;
        R[k] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i) {
        double ks = p->secrete[sp[i]], kap = p->consume[sp[i]];
        if (ks == 0.0 && kap == 0.0) continue;
        int nodes[8][3];
        double w[8];
        int nc = orc_corners(p, pos + i * p->dim, nodes, w);
        for (int m = 0; m < nc; ++m) {
            int64_t g = orc_gidx(p, nodes[m]);
            double vol = orc_tau(p, nodes[m]) * hd;
            S[g] += p->dt * ks * w[m] / vol;
            R[g] += kap * w[m] / vol;
        }
    }
}

/* One forward-Euler substep of Eq. (1d) on the grid with second-order
 * centred differences (Sect. 3.5), substep dt_s = dt/s:
 *   c' = c + dt_s (D_c Lap_h c - gamma c - R c) + S/s.
 * The paper writes the operator as D2 = I - dt Lap; forward Euler needs
 * I + dt D_c Lap, which is the reading taken. Dirichlet nodes keep their
 * value. */
void orc_pde_substep(const orc_params *p, const double *c, const double *S, const double *R, int s,
                     double *c_out)
{
    double dts = p->dt / s;
    int N0 = orc_gdim(p, 0), N1 = orc_gdim(p, 1), N2 = orc_gdim(p, 2);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N2; ++z)
        for (int64_t y = 0; y < N1; ++y)
            for (int64_t x = 0; x < N0; ++x) {
                int k[3] = {(int)x, (int)y, (int)z};
                int64_t g = orc_gidx(p, k);
                int wall = 0;
                for (int a = 0; a < p->dim; ++a)
                    if (k[a] == 0 || k[a] == p->grid[a] - 1) wall = 1;
                if (p->pde_bc == 1 && wall) {
                    c_out[g] = c[g];
                    continue;
                }
                double lap = 0.0;
                for (int a = 0; a < p->dim; ++a) {
                    int kp[3] = {k[0], k[1], k[2]}, km[3] = {k[0], k[1], k[2]};
                    kp[a] = orc_nbr(p, a, k[a] + 1);
                    km[a] = orc_nbr(p, a, k[a] - 1);
                    double h = orc_grid_h(p, a);
                    lap += (c[orc_gidx(p, kp)] - 2.0 * c[g] + c[orc_gidx(p, km)]) / (h * h);
                }
                double rhs = p->Dc * lap - p->gamma * c[g] - (R ? R[g] : 0.0) * c[g];
                c_out[g] = c[g] + dts * rhs + (S ? S[g] : 0.0) / s;
            }
}

/* ------------------------------------------------------------------------ */
/* One time step (order of Sect. 3): drift from c^n at X^n, pair force at   */
/* X^n, Euler-Maruyama move (Eq. (2) with the drift of Eq. (1b)), fixed-step */
/* reactions (Sect. 2.1, 3.4; only if enabled), boundary handling, density  */
/* estimate at X^{n+1}, and the PDE from c^n to c^{n+1}.                     */
/* ------------------------------------------------------------------------ */

/* Reflecting walls (Sect. 3.2): x < lo -> 2 lo - x, x > hi -> 2 hi - x,
 * repeated until inside (the paper reflects once; a large step may need
 * more). Periodic (Sect. 4): wrap into [lo, hi). */
static double orc_boundary(const orc_params *p, int a, double x)
{
    double lo = p->lo[a], hi = p->hi[a], L = hi - lo;
    if (p->boundary == 1) {
        x = lo + (x - lo) - L * floor((x - lo) / L);
        if (x >= hi) x -= L;
        if (x < lo) x = lo;
        return x;
    }
    for (int it = 0; it < 64 && (x < lo || x > hi); ++it) {
        if (x < lo) x = 2.0 * lo - x;
        else if (x > hi) x = 2.0 * hi - x;
    }
    if (x < lo) x = lo;
    if (x > hi) x = hi;
    return x;
}

/* Advances the particles one step: pos (n x dim) and sp (n) in place, ids
 * give the Philox counters, c is read (c^n). disp (n x dim, nullable)
 * accumulates the unwrapped displacement (the `starting` correction of
 * Sect. 4). Optional F_out / drift_out (n x dim) receive the pair force and
 * drift used. */
void orc_move(const orc_params *p, int64_t n, double *pos, uint8_t *sp, const uint32_t *ids,
              const double *c, int64_t step, double *disp, double *F_out, double *drift_out)
{
    int d = p->dim;
    double *F = (double *)malloc(sizeof(double) * (size_t)(n * d + 1));
    double *drift = (double *)malloc(sizeof(double) * (size_t)(n * d + 1));
    double *conc = NULL;
    orc_pair_forces(p, n, pos, sp, 1, F, NULL, NULL, NULL, NULL, NULL);
    orc_drift(p, n, pos, sp, c, drift);
    if (p->reactions) {
        conc = (double *)malloc(sizeof(double) * (size_t)(n + 1));
        orc_conc(p, n, pos, c, conc);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double xi[4];
        orc_normals(p->seed, ids[i], (uint64_t)step, ORC_TAG_MOVE, xi);
        int s = sp[i];
        double amp = sqrt(2.0 * p->D[s] * p->dt);
        /* drift increment: dt a (Euler-Maruyama) or dt a / (1 + dt |a|)
         * (tamed Euler; the paper tames the interaction drift of the alpha
         * equation, here the whole drift, which is that for chi_s = 0) */
        double scale = p->dt;
        if (p->move_scheme == 1) {
            double an = 0.0;
            for (int a = 0; a < d; ++a) {
                double v = F[i * d + a] + drift[i * d + a];
                an += v * v;
            }
            scale = p->dt / (1.0 + p->dt * sqrt(an));
        }
        for (int a = 0; a < d; ++a) {
            double x0 = pos[i * d + a];
            double x1 = x0 + scale * (F[i * d + a] + drift[i * d + a]) + amp * xi[a];
            double xb;
            if (p->boundary == 1) {
                xb = orc_boundary(p, a, x1);
                if (disp) disp[i * d + a] += x1 - x0;
            } else {
                xb = orc_boundary(p, a, x1);
                if (disp) disp[i * d + a] += xb - x0;
            }
            pos[i * d + a] = xb;
        }
        if (p->reactions) {
            /* Sect. 3.4: switch when a uniform falls below rate * dt. */
            uint32_t w[4];
            orc_words(p->seed, ids[i], (uint64_t)step, ORC_TAG_REACT, w);
            double u = orc_uniform(w[0]);
            double prop = (p->react_k0[s] + p->react_kc[s] * conc[i]) * p->dt;
            if (u < prop) sp[i] = (uint8_t)p->react_to[s];
        }
    }
    if (F_out) memcpy(F_out, F, sizeof(double) * (size_t)(n * d));
    if (drift_out) memcpy(drift_out, drift, sizeof(double) * (size_t)(n * d));
    free(F);
    free(drift);
    free(conc);
}

/* Hard-sphere overlap correction (Sect. 3.2): after the move, every pair
 * closer than the contact distance eps_ij = (sigma_i + sigma_j)/2 is pushed
 * apart along the line of centres by twice the penetration depth
 * d_p = eps_ij - d_ij; cell i takes the fraction D_i / (D_i + D_j) of it (one
 * half each when both are immobile). All corrections are computed from the
 * moved positions and applied together, then the boundary rule again. disp
 * (nullable) follows the corrected positions. Coincident cells (d_ij = 0)
 * have no line of centres and are left alone. */
void orc_hard_sphere(const orc_params *p, int64_t n, double *pos, const uint8_t *sp, double *disp)
{
    int d = p->dim;
    double *dx = (double *)calloc((size_t)(n * d + 1), sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double diff[3] = {0, 0, 0}, r2 = 0.0;
            for (int a = 0; a < d; ++a) {
                diff[a] = orc_wrap_delta(p, a, pos[i * d + a] - pos[j * d + a]);
                r2 += diff[a] * diff[a];
            }
            double contact = 0.5 * (p->diameter[sp[i]] + p->diameter[sp[j]]);
            double r = sqrt(r2);
            if (!(r > 0.0) || !(r < contact)) continue;
            double Di = p->D[sp[i]], Dj = p->D[sp[j]];
            double wi = Di + Dj > 0.0 ? Di / (Di + Dj) : 0.5;
            double move = 2.0 * (contact - r) * wi;
            for (int a = 0; a < d; ++a) dx[i * d + a] += move * diff[a] / r;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < d; ++a) {
            double x0 = pos[i * d + a];
            double x1 = x0 + dx[i * d + a];
            double xb = orc_boundary(p, a, x1);
            if (disp) disp[i * d + a] += p->boundary == 1 ? x1 - x0 : xb - x0;
            pos[i * d + a] = xb;
        }
    free(dx);
}

/* Gaussian kernel density estimate of the cell densities at the grid nodes
 * (Sect. 2.3 and the density listing of Sect. 3): node l gets
 * rho_s(p_l) = sum_{i of species s} K_s(p_l - X_i) with
 * K_s(x) = (2 pi sigma_s^2)^(-d/2) exp(-|x|^2 / (2 sigma_s^2)), the bandwidth
 * sigma_s the species' diameter, summed over the cells within kde_range
 * bandwidths (minimum image when periodic). Outputs S_l = dt sum_s k_s
 * rho_s(p_l) and R_l = sum_s kappa_s rho_s(p_l), the forms of orc_deposit. */
void orc_kde_deposit(const orc_params *p, int64_t n, const double *pos, const uint8_t *sp, double *S,
                     double *R)
{
    int d = p->dim;
    int N0 = orc_gdim(p, 0), N1 = orc_gdim(p, 1), N2 = orc_gdim(p, 2);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N2; ++z)
        for (int64_t y = 0; y < N1; ++y)
            for (int64_t x = 0; x < N0; ++x) {
                int k[3] = {(int)x, (int)y, (int)z};
                double node[3] = {0, 0, 0};
                for (int a = 0; a < d; ++a) node[a] = p->lo[a] + k[a] * orc_grid_h(p, a);
                double s_acc = 0.0, r_acc = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    int s = sp[i];
                    double ks = p->secrete[s], kap = p->consume[s];
                    if (ks == 0.0 && kap == 0.0) continue;
                    double sig = p->diameter[s];
                    double r2 = 0.0;
                    for (int a = 0; a < d; ++a) {
                        double dd = orc_wrap_delta(p, a, node[a] - pos[i * d + a]);
                        r2 += dd * dd;
                    }
                    double R = p->kde_range * sig;
                    if (!(r2 < R * R)) continue;
                    double K = pow(2.0 * ORC_PI * sig * sig, -0.5 * d) * exp(-r2 / (2.0 * sig * sig));
                    s_acc += p->dt * ks * K;
                    r_acc += kap * K;
                }
                int64_t g = orc_gidx(p, k);
                S[g] = s_acc;
                R[g] = r_acc;
            }
}

/* Full step: orc_move (and the hard-sphere correction when enabled), then
 * the density estimate at X^{n+1} and the PDE substeps c^n -> c^{n+1} (c in
 * place; needs no grid when chem_mode = 1). */
void orc_step(const orc_params *p, int64_t n, double *pos, uint8_t *sp, const uint32_t *ids,
              double *c, int64_t step, double *disp, double *F_out, double *drift_out)
{
    orc_move(p, n, pos, sp, ids, c, step, disp, F_out, drift_out);
    if (p->hard_sphere) orc_hard_sphere(p, n, pos, sp, disp);
    if (p->chem_mode != 0) return;
    int64_t G = orc_grid_size(p);
    double *S = (double *)malloc(sizeof(double) * (size_t)G);
    double *R = (double *)malloc(sizeof(double) * (size_t)G);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)G);
    if (p->deposit_kernel == 1)
        orc_kde_deposit(p, n, pos, sp, S, R);
    else
        orc_deposit(p, n, pos, sp, S, R);
    int s = orc_substeps(p);
    for (int m = 0; m < s; ++m) {
        orc_pde_substep(p, c, S, R, s, tmp);
        memcpy(c, tmp, sizeof(double) * (size_t)G);
    }
    free(S);
    free(R);
    free(tmp);
}

/* nsteps consecutive steps starting at absolute step index step0. */
void orc_run(const orc_params *p, int64_t n, double *pos, uint8_t *sp, const uint32_t *ids,
             double *c, int64_t step0, int64_t nsteps, double *disp)
{
    for (int64_t k = 0; k < nsteps; ++k) orc_step(p, n, pos, sp, ids, c, step0 + k, disp, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Tangent of a step (forward-mode derivative) with respect to              */
/* theta = (chi, inter, D_0 .. D_{ns-1}), with the noise frozen: every       */
/* operation of orc_step is differentiated where it acts. dpos[(i d + a) P   */
/* + k] = dX_ia / dtheta_k and dc[g P + k] = dc_g / dtheta_k are carried     */
/* from step to step (zero at the start for fixed initial data). The         */
/* piecewise choices (which pairs are inside the cutoff, the grid cell of a */
/* particle, the number of wall reflections) are held, so this is the       */
/* derivative wherever the trajectory is differentiable. The primal state   */
/* is advanced by the functions above, exactly as orc_step does.             */
/* Pieces, in the order of orc_step:                                         */
/*   pair term g(r) u, u = X_i - X_j, g = f(r)/r, f = (inter/eps)(e^{-r/eps} */
/*   - shift): d(g u) = g du + g'(r) (u.du / r) u + (dg/dinter) u dinter;    */
/*   drift chi kappa_s sum_m w_m(X) grad_h c(node_m): the product rule over  */
/*   chi, the weights (dw_m/dx_a = +-1/h_a times the other axes' factors)    */
/*   and c; noise sqrt(2 D_s dt) xi: d/dD_s = dt / sqrt(2 D_s dt) xi; a wall */
/*   reflection negates the tangent, a periodic wrap keeps it; the deposit   */
/*   differentiates the weights; the PDE substep is linear in (c, S) and    */
/*   bilinear in (R, c).                                                     */
/* Columns past 2 + ns carry no parameter: seeded by the caller (a direction */
/* in the initial positions), they give directional derivatives.            */
/* Supported: Euler-Maruyama, cloud-in-cell deposit, no reactions and no    */
/* hard-sphere correction (returns -1 otherwise; -2 for a wrong P).         */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_THETA (2 + ORC_MAX_SPECIES)

typedef struct orc_tan_ctx {
    const orc_params *p;
    const double *pos, *dpos;
    const uint8_t *sp;
    int64_t i;
    int P;
    double dF[3][ORC_MAX_THETA];
} orc_tan_ctx;

static void orc_tan_visit(void *vctx, int64_t j)
{
    orc_tan_ctx *c = (orc_tan_ctx *)vctx;
    if (j == c->i) return;
    const orc_params *p = c->p;
    const int d = p->dim, P = c->P;
    orc_pair_geom g;
    orc_geom(p, c->pos + c->i * d, c->pos + j * d, c->sp[c->i], c->sp[j], &g);
    if (!(g.r > 0.0) || !(g.r < g.rc)) return;
    double e = exp(-g.r / g.eps);
    double shift = p->cutoff_mode == 1 ? exp(-p->cutoff_factor) : 0.0;
    double f = orc_force_mag(p, g.r, g.eps);
    double gr = f / g.r;
    double fp = -p->inter / (g.eps * g.eps) * e;  /* df/dr */
    double gp = (fp * g.r - f) / g.r2;              /* d(f/r)/dr */
    double gi = (e - shift) / (g.eps * g.r);        /* d(f/r)/dinter */
    for (int k = 0; k < P; ++k) {
        double du[3] = {0.0, 0.0, 0.0}, udu = 0.0;
        for (int a = 0; a < d; ++a) {
            du[a] = c->dpos[(c->i * d + a) * P + k] - c->dpos[(j * d + a) * P + k];
            udu += g.d[a] * du[a];
        }
        for (int a = 0; a < d; ++a) {
            double v = gr * du[a] + gp * (udu / g.r) * g.d[a];
            if (k == 1) v += gi * g.d[a];
            c->dF[a][k] += v;
        }
    }
}

/* Derivatives of the interpolation weights of orc_corners: dw[m][a]. */
static void orc_corner_derivs(const orc_params *p, const double *x, double dw[8][3])
{
    int k0[3] = {0, 0, 0}, k1[3] = {0, 0, 0};
    double f[3] = {0, 0, 0};
    for (int a = 0; a < p->dim; ++a) orc_cell_frac(p, a, x[a], &k0[a], &k1[a], &f[a]);
    int nc = 1 << p->dim;
    for (int m = 0; m < nc; ++m)
        for (int a = 0; a < 3; ++a) {
            dw[m][a] = 0.0;
            if (a >= p->dim) continue;
            double v = (((m >> a) & 1) ? 1.0 : -1.0) / orc_grid_h(p, a);
            for (int b = 0; b < p->dim; ++b)
                if (b != a) v *= ((m >> b) & 1) ? f[b] : (1.0 - f[b]);
            dw[m][a] = v;
        }
}

/* Central difference of column k of a tangent grid (dc[g P + k]) at node k3. */
static double orc_node_grad_col(const orc_params *p, const double *dc, int P, int col, const int k3[3], int a)
{
    int kp[3] = {k3[0], k3[1], k3[2]}, km[3] = {k3[0], k3[1], k3[2]};
    kp[a] = orc_nbr(p, a, k3[a] + 1);
    km[a] = orc_nbr(p, a, k3[a] - 1);
    return (dc[orc_gidx(p, kp) * P + col] - dc[orc_gidx(p, km) * P + col]) / (2.0 * orc_grid_h(p, a));
}

/* Reflection sign of orc_boundary at x: +1 or -1 per the parity of the
 * reflections, 1 when periodic, 0 when the position was clamped. */
static double orc_boundary_sign(const orc_params *p, int a, double x)
{
    if (p->boundary == 1) return 1.0;
    double lo = p->lo[a], hi = p->hi[a], sg = 1.0;
    for (int it = 0; it < 64 && (x < lo || x > hi); ++it) {
        if (x < lo) x = 2.0 * lo - x;
        else if (x > hi) x = 2.0 * hi - x;
        sg = -sg;
    }
    return (x < lo || x > hi) ? 0.0 : sg;
}

int orc_step_tangent(const orc_params *p, int64_t n, double *pos, uint8_t *sp, const uint32_t *ids,
                     double *c, int64_t step, int P, double *dpos, double *dc)
{
    if (p->move_scheme != 0 || p->hard_sphere || p->reactions || p->deposit_kernel != 0) return -1;
    if (P < 2 + p->n_species || P > ORC_MAX_THETA) return -2;
    const int d = p->dim;
    double *F = (double *)malloc(sizeof(double) * (size_t)(n * d + 1));
    double *drift = (double *)malloc(sizeof(double) * (size_t)(n * d + 1));
    double *dstep = (double *)calloc((size_t)(n * d * P + 1), sizeof(double));  /* d(F + drift) */
    orc_pair_forces(p, n, pos, sp, 1, F, NULL, NULL, NULL, NULL, NULL);
    orc_drift(p, n, pos, sp, c, drift);
    orc_cells cl;
    memset(&cl, 0, sizeof(cl));
    orc_cells_build(p, n, pos, &cl);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        orc_tan_ctx t;
        memset(&t, 0, sizeof(t));
        t.p = p;
        t.pos = pos;
        t.dpos = dpos;
        t.sp = sp;
        t.i = i;
        t.P = P;
        orc_candidates(p, &cl, n, pos, i, orc_tan_visit, &t);
        /* drift tangent */
        double kap = p->chemotactic[sp[i]];
        double ddr[3][ORC_MAX_THETA];
        memset(ddr, 0, sizeof(ddr));
        if (kap != 0.0) {
            if (p->chem_mode == 1) {
                for (int a = 0; a < d; ++a) ddr[a][0] = kap * p->fixed_grad[a];
            } else {
                int nodes[8][3];
                double w[8], dw[8][3];
                int nc = orc_corners(p, pos + i * d, nodes, w);
                orc_corner_derivs(p, pos + i * d, dw);
                for (int m = 0; m < nc; ++m)
                    for (int a = 0; a < d; ++a) {
                        double gm = orc_node_grad(p, c, nodes[m], a);
                        ddr[a][0] += kap * w[m] * gm;  /* d/dchi */
                        for (int k = 0; k < P; ++k) {
                            double wdx = 0.0;
                            for (int b = 0; b < d; ++b) wdx += dw[m][b] * dpos[(i * d + b) * P + k];
                            double dgm = dc ? orc_node_grad_col(p, dc, P, k, nodes[m], a) : 0.0;
                            ddr[a][k] += p->chi * kap * (wdx * gm + w[m] * dgm);
                        }
                    }
            }
        }
        for (int a = 0; a < d; ++a)
            for (int k = 0; k < P; ++k) dstep[(i * d + a) * P + k] = t.dF[a][k] + ddr[a][k];
    }
    orc_cells_free(&cl);
    /* the move (primal as orc_move) and its tangent */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double xi[4];
        orc_normals(p->seed, ids[i], (uint64_t)step, ORC_TAG_MOVE, xi);
        int s = sp[i];
        double amp = sqrt(2.0 * p->D[s] * p->dt);
        double damp = amp > 0.0 ? p->dt / amp : 0.0;  /* d amp / d D_s */
        for (int a = 0; a < d; ++a) {
            double x0 = pos[i * d + a];
            double x1 = x0 + p->dt * (F[i * d + a] + drift[i * d + a]) + amp * xi[a];
            double sg = orc_boundary_sign(p, a, x1);
            pos[i * d + a] = orc_boundary(p, a, x1);
            for (int k = 0; k < P; ++k) {
                double v = dpos[(i * d + a) * P + k] + p->dt * dstep[(i * d + a) * P + k];
                if (k == 2 + s) v += damp * xi[a];
                dpos[(i * d + a) * P + k] = sg * v;
            }
        }
    }
    free(F);
    free(drift);
    free(dstep);
    if (p->chem_mode != 0) return 0;
    /* deposit at X^{n+1} and its tangent */
    int64_t G = orc_grid_size(p);
    double *S = (double *)malloc(sizeof(double) * (size_t)G);
    double *R = (double *)malloc(sizeof(double) * (size_t)G);
    double *dS = (double *)calloc((size_t)(G * P), sizeof(double));
    double *dR = (double *)calloc((size_t)(G * P), sizeof(double));
    orc_deposit(p, n, pos, sp, S, R);
    double hd = 1.0;
    for (int a = 0; a < d; ++a) hd *= orc_grid_h(p, a);
    for (int64_t i = 0; i < n; ++i) {
        double ks = p->secrete[sp[i]], kap = p->consume[sp[i]];
        if (ks == 0.0 && kap == 0.0) continue;
        int nodes[8][3];
        double w[8], dw[8][3];
        int nc = orc_corners(p, pos + i * d, nodes, w);
        orc_corner_derivs(p, pos + i * d, dw);
        for (int m = 0; m < nc; ++m) {
            int64_t g = orc_gidx(p, nodes[m]);
            double vol = orc_tau(p, nodes[m]) * hd;
            for (int k = 0; k < P; ++k) {
                double wdx = 0.0;
                for (int b = 0; b < d; ++b) wdx += dw[m][b] * dpos[(i * d + b) * P + k];
                dS[g * P + k] += p->dt * ks * wdx / vol;
                dR[g * P + k] += kap * wdx / vol;
            }
        }
    }
    /* PDE substeps c^n -> c^{n+1} and their tangent */
    int ns = orc_substeps(p);
    double dts = p->dt / ns;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)G);
    double *dtmp = (double *)malloc(sizeof(double) * (size_t)(G * P));
    int N0 = orc_gdim(p, 0), N1 = orc_gdim(p, 1), N2 = orc_gdim(p, 2);
    for (int m = 0; m < ns; ++m) {
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < N2; ++z)
            for (int64_t y = 0; y < N1; ++y)
                for (int64_t x = 0; x < N0; ++x) {
                    int k3[3] = {(int)x, (int)y, (int)z};
                    int64_t g = orc_gidx(p, k3);
                    int wall = 0;
                    for (int a = 0; a < d; ++a)
                        if (k3[a] == 0 || k3[a] == p->grid[a] - 1) wall = 1;
                    for (int k = 0; k < P; ++k) {
                        if (p->pde_bc == 1 && wall) {
                            dtmp[g * P + k] = dc[g * P + k];
                            continue;
                        }
                        double lap = 0.0;
                        for (int a = 0; a < d; ++a) {
                            int kp[3] = {k3[0], k3[1], k3[2]}, km[3] = {k3[0], k3[1], k3[2]};
                            kp[a] = orc_nbr(p, a, k3[a] + 1);
                            km[a] = orc_nbr(p, a, k3[a] - 1);
                            double h = orc_grid_h(p, a);
                            lap += (dc[orc_gidx(p, kp) * P + k] - 2.0 * dc[g * P + k] + dc[orc_gidx(p, km) * P + k]) / (h * h);
                        }
                        double rhs = p->Dc * lap - p->gamma * dc[g * P + k] - R[g] * dc[g * P + k] - dR[g * P + k] * c[g];
                        dtmp[g * P + k] = dc[g * P + k] + dts * rhs + dS[g * P + k] / ns;
                    }
                }
        orc_pde_substep(p, c, S, R, ns, tmp);
        memcpy(c, tmp, sizeof(double) * (size_t)G);
        memcpy(dc, dtmp, sizeof(double) * (size_t)(G * P));
    }
    free(S);
    free(R);
    free(dS);
    free(dR);
    free(tmp);
    free(dtmp);
    return 0;
}

/* nsteps tangent steps from absolute step index step0 (see orc_step_tangent). */
int orc_run_tangent(const orc_params *p, int64_t n, double *pos, uint8_t *sp, const uint32_t *ids,
                    double *c, int64_t step0, int64_t nsteps, int P, double *dpos, double *dc)
{
    for (int64_t k = 0; k < nsteps; ++k) {
        int r = orc_step_tangent(p, n, pos, sp, ids, c, step0 + k, P, dpos, dc);
        if (r) return r;
    }
    return 0;
}
