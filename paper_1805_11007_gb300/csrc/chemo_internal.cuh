// chemo_internal.cuh -- device-side definitions shared by the kernels and the
// engine of the GB300 chemotaxis step (arXiv:1805.11007). Not part of the
// public ABI (include/chemo.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace chemo {

constexpr int MAXS = 8;
constexpr uint32_t ID_BITS = 29;                 // particle id in the low 29 bits of .w
constexpr uint32_t ID_MASK = (1u << ID_BITS) - 1u;
constexpr uint32_t SP_SHIFT = ID_BITS;           // species in the top 3 bits

// Latched device error bits (OR-ed into KP::err).
enum : uint32_t {
    ERR_NONFINITE = 1u,
    ERR_DOMAIN = 2u,
    ERR_OVERFLOW = 4u,
    ERR_TIMEOUT = 8u,
    ERR_SPECIES = 16u,
};

// Philox stream tags (third counter word).
constexpr uint32_t TAG_MOVE = 0u;
constexpr uint32_t TAG_REACT = 2u;
constexpr uint32_t TAG_INIT = 3u;   // initial positions (chemo_init_positions)

// Kernel parameter block, passed by value to every kernel.
struct KP {
    // particles and cell list
    int64_t n;
    int dim, periodic, search;  // search 1: 3^d bins >= r_c (warp), 2: 2^d bins >= 2 r_c, 3: 3^d (per lane),
                                // 4: upper half of the 3^d window (per lane, each pair once)
    int warp_runs;              // search 1: warps with at most this many bins search together
    int bt;                     // threads per block of the half-window pair kernel and its move kernel
                                // (128, 256 or 512; the same register budget per thread)
    int pairs;                  // 0: no pair interaction (inter = 0 or zero range)
    float lo[3], hi[3], L[3], halfL[3];
    int nb[3];                  // bins per axis
    float inv_b[3], bside[3];   // nb/L and L/nb per axis
    int px;                     // row pitch of the bin table (nb[0] rounded up to 8)
    int64_t bin_slots;          // px * nb[1] * nb[2]; bins are row-major, x fastest
    int64_t ngroups;            // bin_slots / 8: groups of 8 bins of one row
    // Replicates (2D only): independent simulations of the same model stacked
    // as layers. A particle's layer is its .z (an exact small integer); bins
    // and grid nodes carry the layer as their third index (nb[2] = g[2] =
    // layers), so pairs, gradients and deposits never cross layers. Layer l
    // holds the ids layer_off[l] .. layer_off[l+1]-1 of the caller's arrays,
    // stored in .w as the id local to the layer; its Philox key is seed + l.
    int layers;
    const int64_t *layer_off;    // device, layers + 1 entries (NULL when layers == 1)
    // Sub-domain of a z-slab decomposition (sub = 1): cells with id ID_MASK
    // are ghosts (copies of a neighbour's cells: they exert pair forces but
    // are neither moved nor deposited). open_z bit 0 / 1: the z = lo / hi
    // face is an inner face (no reflection, no half control volume).
    int sub, open_z;
    // species tables (index s * MAXS + t)
    int ns;
    float rc2[MAXS * MAXS];      // r_c,st^2
    float inv_eps[MAXS * MAXS];  // 1/eps_st
    float amp_f[MAXS * MAXS];    // inter/eps_st
    float shift[MAXS * MAXS];    // exp(-cutoff_factor) when force shifted, else 0
    float fq, fq_inv;            // fixed-point quantum of the force sum and its inverse
    float rsp2[MAXS];            // squared search radius of each species (max cutoff, small margin)
    float noise[MAXS];           // sqrt(2 D_s dt)
    float chem[MAXS];            // chi * chemotactic_s
    float chemotactic_f[MAXS];   // chemotactic_s (the multiplier of chi)
    float inter_f;               // interaction strength
    float src[MAXS];             // k_s dt / h^d
    float cons[MAXS];            // kappa_s / h^d
    float rk0[MAXS], rkc[MAXS];  // switching rates
    int rto[MAXS];
    int reactions;
    // variants
    int move_scheme;             // 0 Euler-Maruyama, 1 tamed Euler
    int hard_sphere;             // overlap correction after the move
    float hs_contact[MAXS * MAXS];  // contact distance (sigma_s + sigma_t)/2
    float hs_share[MAXS * MAXS];    // share of the separation taken by the first: D_s/(D_s+D_t)
    int kde;                     // 1: Gaussian kernel density deposit (gathered per node)
    int kde_win;                 // bins searched on each side of a node's bin
    float kde_r2[MAXS];          // squared truncation radius (kde_range sigma_s)^2
    float kde_c[MAXS];           // 1 / (2 sigma_s^2)
    float kde_src[MAXS];         // dt k_s (2 pi sigma_s^2)^(-d/2)
    float kde_cons[MAXS];        // kappa_s (2 pi sigma_s^2)^(-d/2)
    float kde_rmax;              // largest truncation radius over the species
    float kde_qs, kde_qs_inv;    // fixed-point quantum of the source sum (2^-24 of its largest term)
    float kde_qr, kde_qr_inv;    // the same for the consumption sum
    float hgrid[3];              // grid spacing per axis
    double lo_d[3], hgrid_d[3];  // box corner and grid spacing in double (node positions)
    float dt;
    double dt_d;                 // dt in double (switching decision)
    uint32_t seed_lo, seed_hi;
    int chem_mode;               // 0 grid, 1 fixed gradient
    float fixed_g[3];
    // grid
    int has_grid;
    int g[3];
    int64_t G;
    float inv_h[3], inv_2h[3], inv_h2[3];
    int pde_bc;                  // 0 Neumann, 1 Dirichlet, 2 periodic
    float Dc, gamma;
    int substeps;
    float dts;
    int pde_multi;               // 1: 2D grid, several substeps per launch (temporal blocking)
    int pde_launches;            // PDE launches per step (each swaps the c buffers once)
    int zero_src;                // 1: the particle kernel clears the source grids of the last step
    int fused_deposit;           // 1: deposit straight into c^{n+1} (one substep)
    int overlap;                 // 1: PDE concurrent with the particle kernel (second stream)
    // buffers
    float4 *S, *U;               // sorted state, unsorted next state
    uint32_t *slot;              // rank of each U entry inside its bin
    float4 *dS, *dU;             // unwrapped displacement (optional)
    // Cell list, two levels: packed 16-bit counts per bin (2 per word) and the
    // offset of every group of 8 bins. cnt_cur describes the sorted state S;
    // cnt_nxt collects the bins of the state being written to U.
    uint32_t *cnt_cur, *cnt_nxt;
    uint32_t *gstart;            // group offsets (ngroups + 1) of the state last scanned
    unsigned long long *tiles;   // scan tile status
    uint32_t scan_spins;         // polls of the scan's look-back wait before it gives up (ERR_TIMEOUT)
    uint32_t *tile_ctr;          // dynamic tile counter of the scan
    uint32_t *scan_seq;          // scan epoch counter
    float *c[2];                 // chemical ping-pong buffers
    float *srcg, *Rg;            // source and consumption grids (substeps > 1)
    uint32_t *err;               // latched error bits
    unsigned long long *step;    // absolute index of the step being computed
    // non-NULL while profiling: in-cutoff pairs and candidate tests of the
    // half window, each counted into PROF_SLOTS counters (a block adds to
    // slot blockIdx.x mod PROF_SLOTS: one counter for every warp of a launch
    // serialised its atomics and slowed the profiled kernels)
    unsigned long long *pair_count;
    unsigned long long *test_count;
    // adjoint recording (pos == NULL: off): the particle kernel stores, for
    // steps s0 .. s0 + nk - 1 (absolute indices; with period > 0 step s goes
    // to slot (s - s0) mod period, nk = period), the positions before the
    // step and the pair force (by id, [k][id][dim]), the sorted state
    // ([k][n]), its count table and group offsets ([k][cwords], [k][gwords])
    // and the field c^n ([k][G]). With pos_gap > 0 the position slots skip
    // one after every pos_gap steps (room for a segment's final positions).
    struct TapeOut {
        float *pos, *c, *F;
        float4 *S;
        uint32_t *cnt, *gst;
        unsigned long long s0, nk, period, pos_gap;
        int64_t cwords, gwords;
    } tape;
    long long *Fh;               // search mode 4 (set iff pairs and mode 4): pair-force sums in fixed
                                 // point, FhStride per sorted cell; NULL = the full-window search
};

// stride of the half-window force sums (x, y[, z] and padding to 16 bytes)
template <int DIM>
struct FhStride {
    static constexpr int value = DIM == 3 ? 4 : 2;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), written from the
// published definition: ten rounds of the 4x32 Philox S-box, Weyl key bumps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Words of cell `id` (local to its layer) at step `step` on stream `tag`:
// counter (id, step lo, tag, step hi), key (seed + layer) as (lo, hi) words.
__device__ __forceinline__ uint4 cell_words(const KP &kp, uint32_t id, unsigned long long step,
                                            uint32_t tag, uint32_t layer = 0u)
{
    const uint32_t k0 = kp.seed_lo + layer;
    const uint32_t k1 = kp.seed_hi + (k0 < kp.seed_lo ? 1u : 0u);
    return philox4x32_10(make_uint4(id, (uint32_t)step, tag, (uint32_t)(step >> 32)), k0, k1);
}

// u = (w + 1/2) 2^-32 in single precision (never 0).
__device__ __forceinline__ float word_uniform(uint32_t w)
{
    return fmaf((float)w, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

// ln u(w) to single-precision relative accuracy over the whole range. For
// u >= 1/2 the logarithm is taken of 1 + (-(1 - u)) with 1 - u formed from
// the complement of the word (exact up to one rounding); u itself rounded to
// single precision would leave 1 - u with an absolute error of 2^-25 and the
// radius sqrt(-2 ln u) off by up to ~2 % where it is small.
__device__ __forceinline__ float word_log_uniform(uint32_t w)
{
    if (w >= 0x80000000u) return log1pf(-fmaf((float)(~w), 2.3283064365386963e-10f, 1.1641532182693481e-10f));
    return logf(word_uniform(w));
}

// (sin, cos) of 2 pi u(w). The top two bits of w give the quarter turn; the
// angle inside it, pi (f + 1/2) 2^-31 with f the low 30 bits, is folded to at
// most pi/4 with integer arithmetic (pi/2 minus it for f in the upper half),
// so the small one of the two results keeps single-precision relative
// accuracy instead of the 2^-24 absolute error of 2 u rounded near a multiple
// of 1/2.
__device__ __forceinline__ void word_sincos_2pi(uint32_t w, float &s, float &c)
{
    const uint32_t q = w >> 30, f = w & 0x3FFFFFFFu;
    const bool low = f < 0x20000000u;
    const uint32_t k = low ? f : 0x3FFFFFFFu - f;
    float s0, c0;
    sincospif(fmaf((float)k, 4.656612873077393e-10f, 2.3283064365386963e-10f), &s0, &c0);
    const float sa = low ? s0 : c0, ca = low ? c0 : s0;  // sin, cos of the angle inside the quarter
    // rotate by q quarter turns
    s = q == 0 ? sa : (q == 1 ? ca : (q == 2 ? -sa : -ca));
    c = q == 0 ? ca : (q == 1 ? -sa : (q == 2 ? -ca : sa));
}

// Box-Muller transform of the uniform pair (u(a), u(b)): two N(0,1) draws,
// (r cos 2 pi u(b), r sin 2 pi u(b)) with r = sqrt(-2 ln u(a)).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b)
{
    const float r = sqrtf(-2.0f * word_log_uniform(a));
    float s, c;
    word_sincos_2pi(b, s, c);
    return make_float2(r * c, r * s);
}

// ---------------------------------------------------------------------------
// Cell list: FP32 bin rule (no contraction) and bin keys.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bin_axis(float x, float lo, float inv_b, int nb)
{
    const float t = __fmul_rn(__fsub_rn(x, lo), inv_b);
    int c = __float2int_rd(t);
    c = c < 0 ? 0 : c;
    return c > nb - 1 ? nb - 1 : c;
}

__device__ __forceinline__ uint32_t bin_key(const KP &kp, int cx, int cy, int cz)
{
    return (uint32_t)cx + (uint32_t)kp.px * ((uint32_t)cy + (uint32_t)kp.nb[1] * (uint32_t)cz);
}

// Offset of bin k in the sorted arrays: its group's offset plus its offset
// within the group of 8 bins, which the scan writes over the bin's 16-bit
// count (2 per word; the first bin of a group has offset 0).
__device__ __forceinline__ uint32_t bin_start(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ gstart,
                                              uint32_t k)
{
    uint32_t s = __ldg(&gstart[k >> 3]);
    if (k & 7u) s += __ldg(reinterpret_cast<const unsigned short *>(cnt) + k);
    return s;
}

// Largest count of one bin: counts are 16-bit halves of a 32-bit word, so a
// 65536th particle in one bin would carry into the neighbouring bin's count.
constexpr uint32_t BIN_COUNT_MAX = 0xFFFFu;

// Counters per profiling count (KP::pair_count, KP::test_count); a power of two.
constexpr int PROF_SLOTS = 512;

// Counts particle key k into the packed counts (zero before the count; the
// scan turns them into offsets within the group afterwards); returns its
// slot in the bin
// (the count before it). A bin holds at most BIN_COUNT_MAX particles.
__device__ __forceinline__ uint32_t count_bin(uint32_t *cnt, uint32_t k, uint32_t *err)
{
    const uint32_t sh = (k & 1u) * 16u;
    const uint32_t old = atomicAdd(&cnt[k >> 1], 1u << sh);
    const uint32_t slot = (old >> sh) & BIN_COUNT_MAX;
    if (slot == BIN_COUNT_MAX) atomicOr(err, 4u /* ERR_OVERFLOW */);
    return slot;
}

// Layer of a particle (0 unless replicates are stacked), clamped to the table.
__device__ __forceinline__ int layer_of(const KP &kp, float4 p)
{
    if (kp.dim == 3 || kp.layers <= 1) return 0;
    const int l = (int)p.z;
    return l < 0 ? 0 : (l >= kp.layers ? kp.layers - 1 : l);
}

// Index of a particle in the caller's arrays (layer offset + local id).
__device__ __forceinline__ int64_t gid_of(const KP &kp, float4 p)
{
    const int64_t id = __float_as_uint(p.w) & ID_MASK;
    return kp.layers > 1 ? kp.layer_off[layer_of(kp, p)] + id : id;
}

__device__ __forceinline__ void cell_of(const KP &kp, float4 p, int &cx, int &cy, int &cz)
{
    cx = bin_axis(p.x, kp.lo[0], kp.inv_b[0], kp.nb[0]);
    cy = bin_axis(p.y, kp.lo[1], kp.inv_b[1], kp.nb[1]);
    cz = kp.dim == 3 ? bin_axis(p.z, kp.lo[2], kp.inv_b[2], kp.nb[2]) : layer_of(kp, p);
}

__device__ __forceinline__ uint32_t key_of(const KP &kp, float4 p)
{
    int cx, cy, cz;
    cell_of(kp, p, cx, cy, cz);
    return bin_key(kp, cx, cy, cz);
}

// ---------------------------------------------------------------------------
// Grid helpers. Nodes at lo + k h; C-order index x + gx (y + gy z).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t gidx(const KP &kp, int x, int y, int z)
{
    return (int64_t)x + (int64_t)kp.g[0] * ((int64_t)y + (int64_t)kp.g[1] * (int64_t)z);
}

// Neighbour node index with the ghost rule: mirror (walls) or wrap (periodic).
__device__ __forceinline__ int gnbr(const KP &kp, int a, int k)
{
    const int N = kp.g[a];
    if (kp.pde_bc == 2) return k < 0 ? k + N : (k >= N ? k - N : k);
    if (k < 0) return -k;
    if (k > N - 1) return 2 * (N - 1) - k;
    return k;
}

// Grid cell containing x along axis a and the offset in it. The cell
// coordinate t = (x - lo)/h is carried as t_hi + err with err the exact FMA
// residual of the product, so the offset keeps ~2^-24 relative accuracy
// instead of the ~2^-24 N absolute error of a rounded product.
__device__ __forceinline__ void gcell(const KP &kp, int a, float x, int &k0, int &k1, float &f)
{
    const int N = kp.g[a];
    const float rel = x - kp.lo[a];
    const float th = __fmul_rn(rel, kp.inv_h[a]);
    const float err = fmaf(rel, kp.inv_h[a], -th);
    const float fl = floorf(th);
    int k = (int)fl;
    float fr = (th - fl) + err;
    if (fr < 0.f) {
        fr += 1.f;
        k -= 1;
    } else if (fr >= 1.f) {
        fr -= 1.f;
        k += 1;
    }
    if (kp.pde_bc == 2) {
        k = k % N;
        if (k < 0) k += N;
        k0 = k;
        k1 = k + 1 == N ? 0 : k + 1;
        f = fr;
    } else {
        if (k < 0) {
            f = (th - 0.f) + err;   // outside the first cell (x < lo): extrapolate in cell 0
            k = 0;
        } else if (k > N - 2) {
            f = (th - (float)(N - 2)) + err;  // x at (or past) the last node: cell N-2
            k = N - 2;
        } else {
            f = fr;
        }
        k0 = k;
        k1 = k + 1;
    }
}

__device__ __forceinline__ void set_err(const KP &kp, uint32_t bits) { atomicOr(kp.err, bits); }

// ---------------------------------------------------------------------------
// Kernel launchers (kernels.cu). All launch on `st` and return the launch
// status; counts of launched kernels are added to *launches when non-NULL.
// ---------------------------------------------------------------------------
cudaError_t launch_step_particles(const KP &kp, int cur, cudaStream_t st, int *launches);
cudaError_t launch_pack(const KP &kp, const float *pos, const uint8_t *sp, const float *disp,
                        cudaStream_t st, int *launches);
cudaError_t launch_scan(const KP &kp, cudaStream_t st, int *launches);
// Runs the scan with its tile counter started at first_tile (then puts the
// counter back to 0 and advances the scan epoch, as the scatter does), so
// the tiles that look back at the unclaimed ones wait until their limit.
cudaError_t launch_scan_from_tile(const KP &kp, uint32_t first_tile, cudaStream_t st);
// Number of tiles (blocks) of the scan of kp's cell list.
unsigned scan_tiles(const KP &kp);
cudaError_t launch_scatter(const KP &kp, int cur, int advance_step, cudaStream_t st, int *launches);
cudaError_t launch_pde(const KP &kp, int cur, cudaStream_t st, int *launches);
// Substeps per launch of the temporal-blocked 2D PDE kernel (its halo width).
#ifndef CHEMO_PDE_MULTI_MAX
#define CHEMO_PDE_MULTI_MAX 12
#endif
constexpr int PDE_MULTI_MAX = CHEMO_PDE_MULTI_MAX;
// Runs `nsub` substeps of the 2D PDE in one launch from cin to cout (c grids
// of kp); use_src adds the source / consumption grids; avg (nullable)
// receives (avg_first) or accumulates avg_scale times the sum of the
// substeps' input values; tau_mode 1 works on c/tau (trapezoid weights) and
// stores tau times the result (the transposed operator of the mirror-ghost
// Laplacian, for the adjoint).
cudaError_t launch_pde_multi(const KP &kp, const float *cin, float *cout, int nsub, int use_src, float *avg,
                             int avg_first, float avg_scale, int tau_mode, cudaStream_t st);
cudaError_t launch_unsort(const KP &kp, float *pos, uint8_t *sp, float *disp, cudaStream_t st);
cudaError_t launch_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t n, cudaStream_t st);
cudaError_t launch_init_positions(int dim, int periodic, const double *lo, const double *hi, uint64_t seed, int64_t n,
                                  int64_t n_alpha, float sigma_frac, float *pos, uint8_t *sp, cudaStream_t st);
// Sub-domains of a z-slab decomposition (slabs.cu). launch_pack_cells ingests
// kp.n records (two float4 each: x, y, z, tag | dx, dy, dz, 0) into U and
// counts their bins; launch_slab_select appends the sorted state's own cells
// to up to SLAB_TARGETS targets; launch_add adds n floats of src to dst.
constexpr int SLAB_TARGETS = 4;
struct SlabSelect {
    int nt;
    float z0[SLAB_TARGETS], z1[SLAB_TARGETS], own0[SLAB_TARGETS], own1[SLAB_TARGETS];
    float4 *out[SLAB_TARGETS];
    int64_t cap[SLAB_TARGETS];
    unsigned long long *count[SLAB_TARGETS];
};
cudaError_t launch_pack_cells(const KP &kp, const float4 *rec, cudaStream_t st);
cudaError_t launch_slab_select(const KP &kp, const SlabSelect &t, cudaStream_t st);
cudaError_t launch_add(float *dst, const float *src, int64_t n, cudaStream_t st);
cudaError_t launch_stage_bins(const KP &kp, int32_t *cells, cudaStream_t st);
cudaError_t launch_stage_sort(const KP &kp, uint32_t *ids, uint32_t *bin_starts, cudaStream_t st);
cudaError_t launch_stage_forces(const KP &kp, float *F, int32_t *count, unsigned long long *idsum,
                                cudaStream_t st);
cudaError_t launch_stage_drift(const KP &kp, int cur, float *drift, cudaStream_t st);
cudaError_t launch_stage_deposit(const KP &kp, float *S, float *R, cudaStream_t st);
cudaError_t launch_fill(float *p, float v, int64_t n, cudaStream_t st);
cudaError_t launch_hard_sphere(const KP &kp, cudaStream_t st, int *launches);
cudaError_t launch_kde(const KP &kp, float *S, float *R, cudaStream_t st, int *launches);

}  // namespace chemo

struct chemo_params;
// Validated parameter block (layout and constants, no buffers) of n
// particles; sets the thread's last-error message on failure (chemo_capi.cu).
int chemo_internal_build_kp(const chemo_params *params, int64_t n, chemo::KP *out);
int chemo_internal_fail(int status, const char *msg);

namespace chemo {

}  // namespace chemo
