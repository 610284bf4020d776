// kernels.cu -- CUDA kernels (sm_103a) of one time step of the hybrid
// chemotaxis model of Bruna, Maini & Robinson (arXiv:1805.11007).
//
// Per step (Sect. 3 order):
//   k_step     one thread per cell in bin-sorted order: gradient of c^n
//              interpolated to X^n (Sect. 3.6), pair force over the
//              neighbouring bins (Sect. 3.2), Euler-Maruyama move (Eq. (2)),
//              optional fixed-step switching (Sect. 3.4), boundary handling
//              (Sect. 3.2 / Sect. 4), new bin key and its count (cell list,
//              Sect. 2.2 / 3.1).
//   k_pde      explicit step of Eq. (1d) (Sect. 3.5), concurrent with k_step
//              when one substep suffices (both only read c^n).
//   k_scan     exclusive scan of the bin counts (single pass, decoupled
//              look-back with bounded waits); clears the counts.
//   k_scatter  stable placement of the moved cells by bin (counting sort) and
//              the cloud-in-cell deposit of their secretion (Sect. 2.3).
#include "chemo_internal.cuh"

namespace chemo {

constexpr int TPB = 256;

// ---------------------------------------------------------------------------
// Species tables staged in shared memory (indexed by the two species of a
// pair, so a warp with mixed species reads them without serialising).
// ---------------------------------------------------------------------------
struct SmemTables {
    float rc2[MAXS * MAXS];
    float inv_eps[MAXS * MAXS];
    float amp_f[MAXS * MAXS];
    float shift[MAXS * MAXS];
};

__device__ __forceinline__ void load_tables(const KP &kp, SmemTables &t)
{
    for (int i = threadIdx.x; i < MAXS * MAXS; i += blockDim.x) {
        t.rc2[i] = kp.rc2[i];
        t.inv_eps[i] = kp.inv_eps[i];
        t.amp_f[i] = kp.amp_f[i];
        t.shift[i] = kp.shift[i];
    }
}

// ---------------------------------------------------------------------------
// Pair force (Sect. 3.2): F_i = sum_{j != i, 0 < r < r_c,ij}
//   (inter/eps_ij) (exp(-r/eps_ij) - shift) (X_i - X_j)/r
// over the particles of a contiguous range of the sorted array. Each pair
// term is rounded once to a 64-bit fixed-point value (quantum
// max(inter/eps) 2^-40, far below FP32 resolution) and summed exactly, so the
// force does not depend on the order of the particles inside a bin (which
// the atomic slots of the counting sort leave unspecified).
// ---------------------------------------------------------------------------
struct FAcc {
    long long x, y, z;
};

template <int DIM, bool PERIODIC, bool STATS>
__device__ __forceinline__ void accum_range(const KP &kp, const SmemTables &t, uint32_t q0, uint32_t q1,
                                            uint32_t self, float4 me, int sp, FAcc &F, int &count,
                                            unsigned long long &idsum)
{
    const float4 *__restrict__ S = kp.S;
    const int row = sp * MAXS;
    q1 = min(q1, (uint32_t)kp.n);  // bin offsets are trusted only up to n
    for (uint32_t q = q0; q < q1; ++q) {
        const float4 o = __ldg(&S[q]);
        float dx = me.x - o.x, dy = me.y - o.y, dz = DIM == 3 ? me.z - o.z : 0.f;
        if (PERIODIC) {
            // minimum image; the shifted coordinate is subtracted first so
            // the difference of two nearby points is formed exactly
            if (dx > kp.halfL[0]) dx = (me.x - kp.L[0]) - o.x;
            else if (dx < -kp.halfL[0]) dx = me.x - (o.x - kp.L[0]);
            if (dy > kp.halfL[1]) dy = (me.y - kp.L[1]) - o.y;
            else if (dy < -kp.halfL[1]) dy = me.y - (o.y - kp.L[1]);
            if (DIM == 3) {
                if (dz > kp.halfL[2]) dz = (me.z - kp.L[2]) - o.z;
                else if (dz < -kp.halfL[2]) dz = me.z - (o.z - kp.L[2]);
            }
        }
        const float r2 = DIM == 3 ? fmaf(dx, dx, fmaf(dy, dy, dz * dz)) : fmaf(dx, dx, dy * dy);
        const int st = row + (int)(__float_as_uint(o.w) >> SP_SHIFT);
        if (r2 < t.rc2[st] && r2 > 0.f && q != self) {
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            const float f = t.amp_f[st] * (__expf(-r * t.inv_eps[st]) - t.shift[st]);
            const float sq = (f * rinv) * kp.fq_inv;
            F.x += __float2ll_rn(sq * dx);
            F.y += __float2ll_rn(sq * dy);
            if (DIM == 3) F.z += __float2ll_rn(sq * dz);
            if (STATS) {
                count += 1;
                idsum += (unsigned long long)(__float_as_uint(o.w) & ID_MASK);
            }
        }
    }
}

// Neighbouring bins of a particle: 3^d bins around its own (search 1) or
// the 2^d bins on the sides it is closest to (search 2). In row-major order
// the bins of one x-row form one contiguous range of the sorted array.
template <int DIM, bool PERIODIC, bool STATS>
__device__ __forceinline__ float3 pair_force(const KP &kp, const SmemTables &t, uint32_t self, float4 me,
                                             int sp, int &count, unsigned long long &idsum)
{
    FAcc F = {0ll, 0ll, 0ll};
    int c[3], lo[3], hi[3];
    const float pc[3] = {me.x, me.y, me.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= DIM) {
            c[a] = 0;
            lo[a] = 0;
            hi[a] = 0;
            continue;
        }
        c[a] = bin_axis(pc[a], kp.lo[a], kp.inv_b[a], kp.nb[a]);
        if (kp.search == 2) {
            const float tt = __fmul_rn(__fsub_rn(pc[a], kp.lo[a]), kp.inv_b[a]) - (float)c[a];
            if (tt < 0.5f) {
                lo[a] = c[a] - 1;
                hi[a] = c[a];
            } else {
                lo[a] = c[a];
                hi[a] = c[a] + 1;
            }
        } else {
            lo[a] = c[a] - 1;
            hi[a] = c[a] + 1;
        }
        if (!PERIODIC) {
            lo[a] = max(lo[a], 0);
            hi[a] = min(hi[a], kp.nb[a] - 1);
        }
    }
    for (int z = lo[2]; z <= hi[2]; ++z) {
        int zz = z;
        if (PERIODIC && DIM == 3) zz = z < 0 ? z + kp.nb[2] : (z >= kp.nb[2] ? z - kp.nb[2] : z);
        for (int y = lo[1]; y <= hi[1]; ++y) {
            int yy = y;
            if (PERIODIC) yy = y < 0 ? y + kp.nb[1] : (y >= kp.nb[1] ? y - kp.nb[1] : y);
            if (!kp.morton) {
                int x0 = lo[0], x1 = hi[0];
                if (PERIODIC && x0 < 0) {  // wrapped cell on the left, then the rest
                    const uint32_t k = bin_key(kp, kp.nb[0] - 1, yy, zz);
                    accum_range<DIM, PERIODIC, STATS>(kp, t, kp.start[k], kp.start[k + 1], self, me, sp, F,
                                                      count, idsum);
                    x0 = 0;
                }
                if (PERIODIC && x1 >= kp.nb[0]) {
                    const uint32_t k = bin_key(kp, 0, yy, zz);
                    accum_range<DIM, PERIODIC, STATS>(kp, t, kp.start[k], kp.start[k + 1], self, me, sp, F,
                                                      count, idsum);
                    x1 = kp.nb[0] - 1;
                }
                if (x0 <= x1) {
                    const uint32_t k0 = bin_key(kp, x0, yy, zz), k1 = bin_key(kp, x1, yy, zz);
                    accum_range<DIM, PERIODIC, STATS>(kp, t, kp.start[k0], kp.start[k1 + 1], self, me, sp, F,
                                                      count, idsum);
                }
            } else {
                for (int x = lo[0]; x <= hi[0]; ++x) {
                    int xx = x;
                    if (PERIODIC) xx = x < 0 ? x + kp.nb[0] : (x >= kp.nb[0] ? x - kp.nb[0] : x);
                    const uint32_t k = bin_key(kp, xx, yy, zz);
                    accum_range<DIM, PERIODIC, STATS>(kp, t, kp.start[k], kp.start[k + 1], self, me, sp, F,
                                                      count, idsum);
                }
            }
        }
    }
    return make_float3(__ll2float_rn(F.x) * kp.fq, __ll2float_rn(F.y) * kp.fq,
                       DIM == 3 ? __ll2float_rn(F.z) * kp.fq : 0.f);
}

// ---------------------------------------------------------------------------
// Gradient of c interpolated to a point (Sect. 3.5 D1x/D1y central
// differences at the nodes, mirror ghosts at walls, then multilinear
// interpolation, Sect. 3.6). Also returns the interpolated c.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ float3 grad_interp(const KP &kp, const float *__restrict__ c, float4 p, float &cval)
{
    int i[2], j[2], k[2] = {0, 0};
    float fx, fy, fz = 0.f;
    gcell(kp, 0, p.x, i[0], i[1], fx);
    gcell(kp, 1, p.y, j[0], j[1], fy);
    if (DIM == 3) gcell(kp, 2, p.z, k[0], k[1], fz);
    const int im = gnbr(kp, 0, i[0] - 1), ip = gnbr(kp, 0, i[1] + 1);
    const int jm = gnbr(kp, 1, j[0] - 1), jp = gnbr(kp, 1, j[1] + 1);
    constexpr int NZ = DIM == 3 ? 2 : 1;
    // corners C[bz][by][bx] and the nodes one beyond them along each axis
    float C[NZ][2][2], XM[NZ][2], XP[NZ][2], YM[NZ][2], YP[NZ][2], ZM[2][2], ZP[2][2];
#pragma unroll
    for (int bz = 0; bz < NZ; ++bz) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            C[bz][b][0] = __ldg(&c[gidx(kp, i[0], j[b], k[bz])]);
            C[bz][b][1] = __ldg(&c[gidx(kp, i[1], j[b], k[bz])]);
            XM[bz][b] = __ldg(&c[gidx(kp, im, j[b], k[bz])]);
            XP[bz][b] = __ldg(&c[gidx(kp, ip, j[b], k[bz])]);
            YM[bz][b] = __ldg(&c[gidx(kp, i[b], jm, k[bz])]);
            YP[bz][b] = __ldg(&c[gidx(kp, i[b], jp, k[bz])]);
        }
    }
    if (DIM == 3) {
        const int km = gnbr(kp, 2, k[0] - 1), kq = gnbr(kp, 2, k[1] + 1);
#pragma unroll
        for (int by = 0; by < 2; ++by)
#pragma unroll
            for (int bx = 0; bx < 2; ++bx) {
                ZM[by][bx] = __ldg(&c[gidx(kp, i[bx], j[by], km)]);
                ZP[by][bx] = __ldg(&c[gidx(kp, i[bx], j[by], kq)]);
            }
    }
    const float wx[2] = {1.f - fx, fx}, wy[2] = {1.f - fy, fy}, wz[2] = {1.f - fz, fz};
    float3 g = make_float3(0.f, 0.f, 0.f);
    cval = 0.f;
#pragma unroll
    for (int bz = 0; bz < NZ; ++bz)
#pragma unroll
        for (int by = 0; by < 2; ++by)
#pragma unroll
            for (int bx = 0; bx < 2; ++bx) {
                const float w = wx[bx] * wy[by] * (DIM == 3 ? wz[bz] : 1.f);
                // central difference at the corner node: c(k+1) - c(k-1)
                const float gx = bx ? XP[bz][by] - C[bz][by][0] : C[bz][by][1] - XM[bz][by];
                const float gy = by ? YP[bz][bx] - C[bz][0][bx] : C[bz][1][bx] - YM[bz][bx];
                g.x = fmaf(w, gx, g.x);
                g.y = fmaf(w, gy, g.y);
                if (DIM == 3) {
                    const float gz = bz ? ZP[by][bx] - C[0][by][bx] : C[NZ - 1][by][bx] - ZM[by][bx];
                    g.z = fmaf(w, gz, g.z);
                }
                cval = fmaf(w, C[bz][by][bx], cval);
            }
    g.x *= kp.inv_2h[0];
    g.y *= kp.inv_2h[1];
    g.z *= DIM == 3 ? kp.inv_2h[2] : 0.f;
    return g;
}

// ---------------------------------------------------------------------------
// Boundary handling (FP32): reflect until inside (walls) or wrap (periodic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float reflect_axis(float x, float lo, float hi)
{
    for (int it = 0; it < 16 && (x < lo || x > hi); ++it) x = x < lo ? 2.f * lo - x : 2.f * hi - x;
    return fminf(fmaxf(x, lo), hi);
}

__device__ __forceinline__ float wrap_axis(float x, float lo, float hi, float L)
{
    if (x >= hi) x -= L;
    else if (x < lo) x += L;
    if (x >= hi || x < lo) {
        x = x - L * floorf((x - lo) / L);
        if (x >= hi || x < lo) x = lo;
    }
    return x;
}

// ---------------------------------------------------------------------------
// k_step: the particle part of one step.
// ---------------------------------------------------------------------------
template <int DIM, bool PERIODIC>
__global__ void __launch_bounds__(TPB) k_step(KP kp, int cur)
{
    __shared__ SmemTables t;
    load_tables(kp, t);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const unsigned long long step = *kp.step;
    const float4 me = kp.S[j];
    const uint32_t w = __float_as_uint(me.w);
    const uint32_t id = w & ID_MASK;
    int sp = (int)(w >> SP_SHIFT);

    int cnt_unused = 0;
    unsigned long long ids_unused = 0ull;
    float3 F = make_float3(0.f, 0.f, 0.f);
    if (kp.pairs) F = pair_force<DIM, PERIODIC, false>(kp, t, (uint32_t)j, me, sp, cnt_unused, ids_unused);

    float3 dr = make_float3(0.f, 0.f, 0.f);
    float conc = 0.f;
    const float chem = kp.chem[sp];
    if (kp.chem_mode == 1) {
        dr = make_float3(chem * kp.fixed_g[0], chem * kp.fixed_g[1], chem * kp.fixed_g[2]);
        if (kp.reactions)
            conc = kp.fixed_g[0] * (me.x - kp.lo[0]) + kp.fixed_g[1] * (me.y - kp.lo[1]) +
                   (DIM == 3 ? kp.fixed_g[2] * (me.z - kp.lo[2]) : 0.f);
    } else if (kp.has_grid && (chem != 0.f || kp.reactions)) {
        const float3 g = grad_interp<DIM>(kp, kp.c[cur], me, conc);
        dr = make_float3(chem * g.x, chem * g.y, chem * g.z);
    }

    // Euler-Maruyama move, Eq. (2) with the drift of Eq. (1b)
    const uint4 rw = cell_words(kp, id, step, TAG_MOVE);
    const float2 n01 = box_muller(rw.x, rw.y);
    float n2 = 0.f;
    if (DIM == 3) n2 = box_muller(rw.z, rw.w).x;
    const float amp = kp.noise[sp];
    const float x1 = me.x + kp.dt * (F.x + dr.x) + amp * n01.x;
    const float y1 = me.y + kp.dt * (F.y + dr.y) + amp * n01.y;
    const float z1 = DIM == 3 ? me.z + kp.dt * (F.z + dr.z) + amp * n2 : 0.f;

    // fixed-step switching (Sect. 3.4): switch when u < rate dt. The
    // comparison that decides the species is taken in double precision, the
    // precision of the paper's code; u = (w + 1/2) 2^-32 is exact there.
    if (kp.reactions) {
        const uint4 rr = cell_words(kp, id, step, TAG_REACT);
        const double u = ((double)rr.x + 0.5) * 2.3283064365386963e-10;
        const double prop = ((double)kp.rk0[sp] + (double)kp.rkc[sp] * (double)conc) * kp.dt_d;
        if (u < prop) sp = kp.rto[sp];
    }

    float xb, yb, zb;
    if (PERIODIC) {
        xb = wrap_axis(x1, kp.lo[0], kp.hi[0], kp.L[0]);
        yb = wrap_axis(y1, kp.lo[1], kp.hi[1], kp.L[1]);
        zb = DIM == 3 ? wrap_axis(z1, kp.lo[2], kp.hi[2], kp.L[2]) : 0.f;
    } else {
        xb = reflect_axis(x1, kp.lo[0], kp.hi[0]);
        yb = reflect_axis(y1, kp.lo[1], kp.hi[1]);
        zb = DIM == 3 ? reflect_axis(z1, kp.lo[2], kp.hi[2]) : 0.f;
    }
    const bool finite = isfinite(x1) && isfinite(y1) && (DIM == 2 || isfinite(z1));
    if (!finite) {
        set_err(kp, ERR_NONFINITE);
        xb = me.x;
        yb = me.y;
        zb = me.z;
    }
    if (kp.dS) {
        float4 d = kp.dS[j];
        if (finite) {
            if (PERIODIC) {
                d.x += x1 - me.x;
                d.y += y1 - me.y;
                d.z += DIM == 3 ? z1 - me.z : 0.f;
            } else {
                d.x += xb - me.x;
                d.y += yb - me.y;
                d.z += DIM == 3 ? zb - me.z : 0.f;
            }
        }
        kp.dU[j] = d;
    }
    const float4 nu = make_float4(xb, yb, zb, __uint_as_float(id | ((uint32_t)sp << SP_SHIFT)));
    kp.U[j] = nu;
    kp.slot[j] = atomicAdd(&kp.cnt[key_of(kp, nu)], 1u);
}

// ---------------------------------------------------------------------------
// k_pack: ingest caller positions (ids = array index) into U and count bins.
// ---------------------------------------------------------------------------
__global__ void k_pack(KP kp, const float *__restrict__ pos, const uint8_t *__restrict__ sp_in,
                       const float *__restrict__ disp)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= kp.n) return;
    float x[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < kp.dim; ++a) {
        float v = pos[i * kp.dim + a];
        if (!isfinite(v)) {
            set_err(kp, ERR_NONFINITE);
            v = kp.lo[a];
        }
        if (v < kp.lo[a] || v > kp.hi[a]) {
            set_err(kp, ERR_DOMAIN);
            v = fminf(fmaxf(v, kp.lo[a]), kp.hi[a]);
        }
        if (kp.periodic && v >= kp.hi[a]) v = kp.lo[a];  // hi is the image of lo
        x[a] = v;
    }
    uint32_t s = sp_in[i];
    if ((int)s >= kp.ns) {
        set_err(kp, ERR_SPECIES);
        s = 0;
    }
    const float4 u = make_float4(x[0], x[1], x[2], __uint_as_float((uint32_t)i | (s << SP_SHIFT)));
    kp.U[i] = u;
    if (kp.dU) {
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (disp) {
            d.x = disp[i * kp.dim + 0];
            d.y = disp[i * kp.dim + 1];
            if (kp.dim == 3) d.z = disp[i * kp.dim + 2];
        }
        kp.dU[i] = d;
    }
    kp.slot[i] = atomicAdd(&kp.cnt[key_of(kp, u)], 1u);
}

// ---------------------------------------------------------------------------
// k_scan: exclusive scan of cnt[0, bin_slots) into start[0, bin_slots]
// (start[bin_slots] = n), clearing cnt. Single pass with decoupled look-back
// (Merrill & Garland, 2016): tiles are claimed in order from an atomic
// counter, each publishes its aggregate, then its inclusive prefix once its
// predecessors' are known. Waits are bounded; a wait that runs out latches
// ERR_TIMEOUT and proceeds.
// ---------------------------------------------------------------------------
constexpr int SCAN_ITEMS = 4;                       // per thread per round
constexpr int SCAN_ROUNDS = 4;
constexpr int SCAN_TILE = TPB * SCAN_ITEMS * SCAN_ROUNDS;  // 4096 bins
constexpr unsigned long long ST_AGG = 1ull, ST_INC = 2ull;
constexpr int ST_VAL_BITS = 38;
constexpr unsigned long long ST_VAL_MASK = (1ull << ST_VAL_BITS) - 1ull;

__device__ __forceinline__ unsigned long long st_pack(uint32_t epoch, unsigned long long flag,
                                                      unsigned long long v)
{
    return ((unsigned long long)epoch << 40) | (flag << ST_VAL_BITS) | (v & ST_VAL_MASK);
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// the block total.
__device__ __forceinline__ uint32_t block_exscan(uint32_t v, uint32_t &total, uint32_t *warp_sums)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < TPB / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < TPB / 32) warp_sums[lane] = s;  // inclusive
    }
    __syncthreads();
    total = warp_sums[TPB / 32 - 1];
    const uint32_t before = wid ? warp_sums[wid - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(TPB) k_scan(KP kp)
{
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_warp[TPB / 32];
    __shared__ unsigned long long s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(kp.tile_ctr, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= gridDim.x) {  // counter not reset: refuse rather than index past the tile table
        if (threadIdx.x == 0) set_err(kp, ERR_OVERFLOW);
        return;
    }
    const uint32_t epoch = (*(volatile uint32_t *)kp.scan_seq % 0xFFFFFFu) + 1u;
    const int64_t B = kp.bin_slots;
    const int64_t base = (int64_t)tile * SCAN_TILE;

    uint32_t v[SCAN_ROUNDS][SCAN_ITEMS];
    uint32_t tsum[SCAN_ROUNDS];
#pragma unroll
    for (int r = 0; r < SCAN_ROUNDS; ++r) {
        const int64_t i0 = base + (int64_t)r * TPB * SCAN_ITEMS + (int64_t)threadIdx.x * SCAN_ITEMS;
        if (i0 + SCAN_ITEMS <= B) {
            const uint4 q = *reinterpret_cast<const uint4 *>(&kp.cnt[i0]);
            v[r][0] = q.x; v[r][1] = q.y; v[r][2] = q.z; v[r][3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < SCAN_ITEMS; ++k) v[r][k] = (i0 + k < B) ? kp.cnt[i0 + k] : 0u;
        }
        tsum[r] = v[r][0] + v[r][1] + v[r][2] + v[r][3];
    }
    uint32_t rpre[SCAN_ROUNDS], rtot[SCAN_ROUNDS];
#pragma unroll
    for (int r = 0; r < SCAN_ROUNDS; ++r) rpre[r] = block_exscan(tsum[r], rtot[r], s_warp);
    uint32_t tile_total = 0;
#pragma unroll
    for (int r = 0; r < SCAN_ROUNDS; ++r) tile_total += rtot[r];

    // publish and look back
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0)
            atomicExch(&kp.tiles[tile], st_pack(epoch, tile == 0 ? ST_INC : ST_AGG, tile_total));
        unsigned long long excl = 0ull;
        int64_t idx = (int64_t)tile - 1;
        bool timed_out = false;
        while (idx >= 0) {
            const int64_t p = idx - lane;
            unsigned long long stw = 0ull;
            unsigned long long flag = ST_INC, val = 0ull;
            if (p >= 0) {
                int spins = 0;
                for (;;) {
                    stw = *(volatile unsigned long long *)&kp.tiles[p];
                    const uint32_t e = (uint32_t)(stw >> 40);
                    flag = (stw >> ST_VAL_BITS) & 3ull;
                    if (e == epoch && flag != 0ull) break;
                    if (++spins > (1 << 22)) {  // bounded wait
                        timed_out = true;
                        flag = ST_INC;
                        stw = 0ull;
                        break;
                    }
                    __nanosleep(32);
                }
                val = stw & ST_VAL_MASK;
            }
            const unsigned inc_mask = __ballot_sync(0xffffffffu, flag == ST_INC);
            const int first = __ffs(inc_mask) - 1;  // nearest predecessor with an inclusive prefix
            unsigned long long contrib = (inc_mask == 0u || lane <= first) ? val : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, o);
            contrib = __shfl_sync(0xffffffffu, contrib, 0);
            excl += contrib;
            if (inc_mask != 0u) break;
            idx -= 32;
        }
        if (timed_out) set_err(kp, ERR_TIMEOUT);
        if (lane == 0) {
            if (tile != 0) {
                __threadfence();
                atomicExch(&kp.tiles[tile], st_pack(epoch, ST_INC, excl + tile_total));
            }
            s_prefix = excl;
        }
    }
    __syncthreads();
    const uint32_t tile_prefix = (uint32_t)s_prefix;
    uint32_t off = tile_prefix;
#pragma unroll
    for (int r = 0; r < SCAN_ROUNDS; ++r) {
        const int64_t i0 = base + (int64_t)r * TPB * SCAN_ITEMS + (int64_t)threadIdx.x * SCAN_ITEMS;
        uint32_t run = off + rpre[r];
        uint32_t out[SCAN_ITEMS];
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            out[k] = run;
            run += v[r][k];
        }
        if (i0 + SCAN_ITEMS <= B) {
            *reinterpret_cast<uint4 *>(&kp.start[i0]) = make_uint4(out[0], out[1], out[2], out[3]);
            *reinterpret_cast<uint4 *>(&kp.cnt[i0]) = make_uint4(0u, 0u, 0u, 0u);
        } else {
#pragma unroll
            for (int k = 0; k < SCAN_ITEMS; ++k)
                if (i0 + k < B) {
                    kp.start[i0 + k] = out[k];
                    kp.cnt[i0 + k] = 0u;
                }
        }
        off += rtot[r];
    }
    if (base + SCAN_TILE >= B && base < B && threadIdx.x == 0) kp.start[B] = tile_prefix + tile_total;
}

// ---------------------------------------------------------------------------
// Cloud-in-cell deposit of one cell (Sect. 2.3): weights w_k of the 2^d nodes
// around x, mass over the node's control volume tau_k h^d (tau = 1/2 per wall
// axis). fused: add S - dt R c^n straight into c^{n+1}; else add to S and R.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void deposit_cic(const KP &kp, float4 u, int sp, float *tS, float *tR,
                                            const float *__restrict__ cin, bool fused)
{
    const float ks = kp.src[sp], kc = kp.cons[sp];
    if (ks == 0.f && kc == 0.f) return;
    int i0, i1, j0, j1, k0 = 0, k1 = 0;
    float fx, fy, fz = 0.f;
    gcell(kp, 0, u.x, i0, i1, fx);
    gcell(kp, 1, u.y, j0, j1, fy);
    if (DIM == 3) gcell(kp, 2, u.z, k0, k1, fz);
    const bool walls = kp.pde_bc != 2;
#pragma unroll
    for (int m = 0; m < (1 << DIM); ++m) {
        const int bx = m & 1, by = (m >> 1) & 1, bz = (m >> 2) & 1;
        const int x = bx ? i1 : i0, y = by ? j1 : j0, z = bz ? k1 : k0;
        float wgt = (bx ? fx : 1.f - fx) * (by ? fy : 1.f - fy);
        if (DIM == 3) wgt *= bz ? fz : 1.f - fz;
        if (walls) {
            if (x == 0 || x == kp.g[0] - 1) wgt *= 2.f;
            if (y == 0 || y == kp.g[1] - 1) wgt *= 2.f;
            if (DIM == 3 && (z == 0 || z == kp.g[2] - 1)) wgt *= 2.f;
        }
        const int64_t g = gidx(kp, x, y, z);
        if (fused) {
            float a = ks * wgt;
            if (kc != 0.f) a -= kp.dt * kc * wgt * __ldg(&cin[g]);
            atomicAdd(&tS[g], a);
        } else {
            if (ks != 0.f) atomicAdd(&tS[g], ks * wgt);
            if (kc != 0.f) atomicAdd(&tR[g], kc * wgt);
        }
    }
}

// ---------------------------------------------------------------------------
// k_scatter: counting-sort placement S[start[key] + slot] = U and the deposit.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(TPB) k_scatter(KP kp, int cur, int advance)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *kp.tile_ctr = 0u;
        *kp.scan_seq += 1u;
        if (advance) *kp.step += 1ull;
    }
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 u = kp.U[j];
    const uint32_t dst = kp.start[key_of(kp, u)] + kp.slot[j];
    if ((int64_t)dst >= kp.n) {
        set_err(kp, ERR_OVERFLOW);
        return;
    }
    kp.S[dst] = u;
    if (kp.dS) kp.dS[dst] = kp.dU[j];
    if (advance && kp.has_grid && kp.chem_mode == 0) {
        const int sp = (int)(__float_as_uint(u.w) >> SP_SHIFT);
        if (kp.fused_deposit)
            deposit_cic<DIM>(kp, u, sp, kp.c[cur ^ 1], nullptr, kp.c[cur], true);
        else
            deposit_cic<DIM>(kp, u, sp, kp.srcg, kp.Rg, nullptr, false);
    }
}

// ---------------------------------------------------------------------------
// k_pde: one substep of Eq. (1d), c' = c + dt_s (D_c Lap_h c - gamma c - R c)
// + S/s (Sect. 3.5). Thread per node, x fastest. Dirichlet wall nodes keep
// their value. On the last substep S and R are cleared after use.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(128) k_pde(KP kp, const float *__restrict__ cin, float *__restrict__ cout,
                                             int use_src, int last)
{
    const int x = blockIdx.x * 128 + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= kp.g[0]) return;
    const int64_t g = gidx(kp, x, y, z);
    const float c0 = cin[g];
    if (kp.pde_bc == 1) {
        bool wall = x == 0 || x == kp.g[0] - 1 || y == 0 || y == kp.g[1] - 1;
        if (DIM == 3) wall = wall || z == 0 || z == kp.g[2] - 1;
        if (wall) {
            cout[g] = c0;
            if (use_src && last) {
                kp.srcg[g] = 0.f;
                kp.Rg[g] = 0.f;
            }
            return;
        }
    }
    const float cxm = __ldg(&cin[gidx(kp, gnbr(kp, 0, x - 1), y, z)]);
    const float cxp = __ldg(&cin[gidx(kp, gnbr(kp, 0, x + 1), y, z)]);
    const float cym = __ldg(&cin[gidx(kp, x, gnbr(kp, 1, y - 1), z)]);
    const float cyp = __ldg(&cin[gidx(kp, x, gnbr(kp, 1, y + 1), z)]);
    float lap = (cxm - 2.f * c0 + cxp) * kp.inv_h2[0] + (cym - 2.f * c0 + cyp) * kp.inv_h2[1];
    if (DIM == 3) {
        const float czm = __ldg(&cin[gidx(kp, x, y, gnbr(kp, 2, z - 1))]);
        const float czp = __ldg(&cin[gidx(kp, x, y, gnbr(kp, 2, z + 1))]);
        lap += (czm - 2.f * c0 + czp) * kp.inv_h2[2];
    }
    float rhs = kp.Dc * lap - kp.gamma * c0;
    float add = 0.f;
    if (use_src) {
        rhs -= kp.Rg[g] * c0;
        add = kp.srcg[g] / (float)kp.substeps;
        if (last) {
            kp.srcg[g] = 0.f;
            kp.Rg[g] = 0.f;
        }
    }
    cout[g] = c0 + kp.dts * rhs + add;
}

// ---------------------------------------------------------------------------
// Read-out and stage kernels.
// ---------------------------------------------------------------------------
__global__ void k_unsort(KP kp, float *__restrict__ pos, uint8_t *__restrict__ sp, float *__restrict__ disp)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 u = kp.S[j];
    const uint32_t w = __float_as_uint(u.w);
    const int64_t id = w & ID_MASK;
    if (id >= kp.n) {
        set_err(kp, ERR_OVERFLOW);
        return;
    }
    if (pos) {
        pos[id * kp.dim + 0] = u.x;
        pos[id * kp.dim + 1] = u.y;
        if (kp.dim == 3) pos[id * kp.dim + 2] = u.z;
    }
    if (sp) sp[id] = (uint8_t)(w >> SP_SHIFT);
    if (disp && kp.dS) {
        const float4 d = kp.dS[j];
        disp[id * kp.dim + 0] = d.x;
        disp[id * kp.dim + 1] = d.y;
        if (kp.dim == 3) disp[id * kp.dim + 2] = d.z;
    }
}

__global__ void k_philox(uint32_t seed_lo, uint32_t seed_hi, const uint4 *__restrict__ ctr, uint4 *__restrict__ out,
                         int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], seed_lo, seed_hi);
}

__global__ void k_stage_bins(KP kp, int32_t *__restrict__ cells)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 u = kp.S[j];
    const int64_t id = __float_as_uint(u.w) & ID_MASK;
    if (id >= kp.n) {
        set_err(kp, ERR_OVERFLOW);
        return;
    }
    int cx, cy, cz;
    cell_of(kp, u, cx, cy, cz);
    cells[id * kp.dim + 0] = cx;
    cells[id * kp.dim + 1] = cy;
    if (kp.dim == 3) cells[id * kp.dim + 2] = cz;
}

__global__ void k_stage_sort(KP kp, uint32_t *__restrict__ ids)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j < kp.n) ids[j] = __float_as_uint(kp.S[j].w) & ID_MASK;
}

template <int DIM, bool PERIODIC>
__global__ void __launch_bounds__(TPB) k_stage_forces(KP kp, float *__restrict__ F_out, int32_t *__restrict__ count,
                                                      unsigned long long *__restrict__ idsum)
{
    __shared__ SmemTables t;
    load_tables(kp, t);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 me = kp.S[j];
    const uint32_t w = __float_as_uint(me.w);
    const int64_t id = w & ID_MASK;
    if (id >= kp.n) {
        set_err(kp, ERR_OVERFLOW);
        return;
    }
    int cnt = 0;
    unsigned long long ids = 0ull;
    float3 F = make_float3(0.f, 0.f, 0.f);
    if (kp.pairs) F = pair_force<DIM, PERIODIC, true>(kp, t, (uint32_t)j, me, (int)(w >> SP_SHIFT), cnt, ids);
    F_out[id * DIM + 0] = F.x;
    F_out[id * DIM + 1] = F.y;
    if (DIM == 3) F_out[id * DIM + 2] = F.z;
    if (count) count[id] = cnt;
    if (idsum) idsum[id] = ids;
}

template <int DIM>
__global__ void k_stage_drift(KP kp, int cur, float *__restrict__ out)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 me = kp.S[j];
    const uint32_t w = __float_as_uint(me.w);
    const int64_t id = w & ID_MASK;
    if (id >= kp.n) {
        set_err(kp, ERR_OVERFLOW);
        return;
    }
    const int sp = (int)(w >> SP_SHIFT);
    const float chem = kp.chem[sp];
    float3 dr = make_float3(0.f, 0.f, 0.f);
    if (kp.chem_mode == 1) {
        dr = make_float3(chem * kp.fixed_g[0], chem * kp.fixed_g[1], chem * kp.fixed_g[2]);
    } else if (kp.has_grid && chem != 0.f) {
        float cv;
        const float3 g = grad_interp<DIM>(kp, kp.c[cur], me, cv);
        dr = make_float3(chem * g.x, chem * g.y, chem * g.z);
    }
    out[id * DIM + 0] = dr.x;
    out[id * DIM + 1] = dr.y;
    if (DIM == 3) out[id * DIM + 2] = dr.z;
}

template <int DIM>
__global__ void k_stage_deposit(KP kp, float *S, float *R)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 u = kp.S[j];
    deposit_cic<DIM>(kp, u, (int)(__float_as_uint(u.w) >> SP_SHIFT), S, R, nullptr, false);
}

__global__ void k_fill(float *p, float v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i < n) p[i] = v;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

cudaError_t launch_step_particles(const KP &kp, int cur, cudaStream_t st, int *launches)
{
    if (kp.n == 0) return cudaSuccess;
    const unsigned nb = blocks_for(kp.n);
    if (kp.dim == 2) {
        if (kp.periodic) k_step<2, true><<<nb, TPB, 0, st>>>(kp, cur);
        else k_step<2, false><<<nb, TPB, 0, st>>>(kp, cur);
    } else {
        if (kp.periodic) k_step<3, true><<<nb, TPB, 0, st>>>(kp, cur);
        else k_step<3, false><<<nb, TPB, 0, st>>>(kp, cur);
    }
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_pack(const KP &kp, const float *pos, const uint8_t *sp, const float *disp, cudaStream_t st,
                        int *launches)
{
    if (kp.n == 0) return cudaSuccess;
    k_pack<<<blocks_for(kp.n), TPB, 0, st>>>(kp, pos, sp, disp);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_scan(const KP &kp, cudaStream_t st, int *launches)
{
    const unsigned tiles = (unsigned)((kp.bin_slots + SCAN_TILE - 1) / SCAN_TILE);
    k_scan<<<tiles, TPB, 0, st>>>(kp);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_scatter(const KP &kp, int cur, int advance, cudaStream_t st, int *launches)
{
    const unsigned nb = kp.n ? blocks_for(kp.n) : 1u;  // one block still resets the scan state
    if (kp.dim == 2) k_scatter<2><<<nb, TPB, 0, st>>>(kp, cur, advance);
    else k_scatter<3><<<nb, TPB, 0, st>>>(kp, cur, advance);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_pde(const KP &kp, int cur, cudaStream_t st, int *launches)
{
    if (!kp.has_grid || kp.chem_mode != 0) return cudaSuccess;
    const dim3 grid((kp.g[0] + 127) / 128, kp.g[1], kp.dim == 3 ? kp.g[2] : 1);
    const int s = kp.substeps;
    const int use_src = kp.fused_deposit ? 0 : 1;
    int c = cur;
    for (int m = 0; m < s; ++m) {
        const int last = m == s - 1;
        if (kp.dim == 2) k_pde<2><<<grid, 128, 0, st>>>(kp, kp.c[c], kp.c[c ^ 1], use_src, last);
        else k_pde<3><<<grid, 128, 0, st>>>(kp, kp.c[c], kp.c[c ^ 1], use_src, last);
        c ^= 1;
        if (launches) ++*launches;
    }
    return cudaGetLastError();
}

cudaError_t launch_unsort(const KP &kp, float *pos, uint8_t *sp, float *disp, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    k_unsort<<<blocks_for(kp.n), TPB, 0, st>>>(kp, pos, sp, disp);
    return cudaGetLastError();
}

cudaError_t launch_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_philox<<<blocks_for(n), TPB, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32),
                                            reinterpret_cast<const uint4 *>(ctr), reinterpret_cast<uint4 *>(out), n);
    return cudaGetLastError();
}

cudaError_t launch_stage_bins(const KP &kp, int32_t *cells, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    k_stage_bins<<<blocks_for(kp.n), TPB, 0, st>>>(kp, cells);
    return cudaGetLastError();
}

cudaError_t launch_stage_sort(const KP &kp, uint32_t *ids, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    k_stage_sort<<<blocks_for(kp.n), TPB, 0, st>>>(kp, ids);
    return cudaGetLastError();
}

cudaError_t launch_stage_forces(const KP &kp, float *F, int32_t *count, unsigned long long *idsum, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    const unsigned nb = blocks_for(kp.n);
    if (kp.dim == 2) {
        if (kp.periodic) k_stage_forces<2, true><<<nb, TPB, 0, st>>>(kp, F, count, idsum);
        else k_stage_forces<2, false><<<nb, TPB, 0, st>>>(kp, F, count, idsum);
    } else {
        if (kp.periodic) k_stage_forces<3, true><<<nb, TPB, 0, st>>>(kp, F, count, idsum);
        else k_stage_forces<3, false><<<nb, TPB, 0, st>>>(kp, F, count, idsum);
    }
    return cudaGetLastError();
}

cudaError_t launch_stage_drift(const KP &kp, int cur, float *drift, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    if (kp.dim == 2) k_stage_drift<2><<<blocks_for(kp.n), TPB, 0, st>>>(kp, cur, drift);
    else k_stage_drift<3><<<blocks_for(kp.n), TPB, 0, st>>>(kp, cur, drift);
    return cudaGetLastError();
}

cudaError_t launch_stage_deposit(const KP &kp, float *S, float *R, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    if (kp.dim == 2) k_stage_deposit<2><<<blocks_for(kp.n), TPB, 0, st>>>(kp, S, R);
    else k_stage_deposit<3><<<blocks_for(kp.n), TPB, 0, st>>>(kp, S, R);
    return cudaGetLastError();
}

cudaError_t launch_fill(float *p, float v, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_fill<<<blocks_for(n), TPB, 0, st>>>(p, v, n);
    return cudaGetLastError();
}

}  // namespace chemo
