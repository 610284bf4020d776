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
#include <cmath>

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
//   (inter/eps_ij) (exp(-r/eps_ij) - shift) (X_i - X_j)/r.
// Each pair term is rounded once to a 64-bit fixed-point value (quantum
// max(inter/eps) 2^-40, far below FP32 resolution) and summed exactly, so the
// force does not depend on the order of the particles inside a bin (which
// the atomic slots of the counting sort leave unspecified).
// ---------------------------------------------------------------------------
struct FAcc {
    long long x, y, z;
};

// ---------------------------------------------------------------------------
// Search window. Bins are stored row-major (x fastest), so the bins of one
// x-row of the window are one contiguous range of the sorted array: the
// window is at most 3^(d-1) ranges (twice that when a periodic row wraps).
// Rows (and the end bins of a row) farther from the particle than its
// species' largest cutoff are skipped. Each thread stages its ranges in
// shared memory and walks all of them in one flattened loop (the warp waits
// for its longest candidate list only, not for the longest bin of every row).
// Candidates inside the cutoff are listed in shared memory; whenever one lane
// of the warp has filled its list, the whole warp evaluates its lists
// together (a mostly converged loop), and once more at the end.
//
// Pair terms are quantised to 32-bit fixed point (quantum 2^-25 of the
// largest pair force, far below FP32 resolution of the sum's tolerance) and
// summed exactly: in int32 over one list (at most LIST_CAP terms, no
// overflow), then in int64. The force is then independent of the order of
// the particles inside a bin (which the atomic slots of the counting sort
// leave unspecified), and no 64-bit conversion runs per pair (those use the
// narrow FP64 pipe).
// ---------------------------------------------------------------------------
// Compile-time tunables of the pair kernels: resident blocks per SM (their
// register budget is 65536 / (256 x blocks)) and the per-lane list length.
#ifndef CHEMO_PAIR_BLOCKS
#define CHEMO_PAIR_BLOCKS 4
#endif
#ifndef CHEMO_LIST_CAP
#define CHEMO_LIST_CAP 24
#endif
constexpr int LIST_CAP = CHEMO_LIST_CAP;  // flushed once a lane holds more than LIST_CAP - UNROLL
#ifndef CHEMO_UNROLL
#define CHEMO_UNROLL 8
#endif
#ifndef CHEMO_BATCH_LOADS
#define CHEMO_BATCH_LOADS 1
#endif
constexpr int UNROLL = CHEMO_UNROLL;  // candidates per lane between two warp votes

template <int DIM, bool PERIODIC>
struct RowCap {
    static constexpr int value = (DIM == 3 ? 9 : 3) * (PERIODIC ? 2 : 1);
};

template <int DIM, bool PERIODIC>
__device__ __forceinline__ void pair_delta(const KP &kp, float4 me, float4 o, float &dx, float &dy, float &dz, float &r2)
{
    dx = me.x - o.x;
    dy = me.y - o.y;
    dz = DIM == 3 ? me.z - o.z : 0.f;
    if (PERIODIC) {
        // minimum image; the shifted coordinate is subtracted first so the
        // difference of two nearby points is formed exactly
        if (dx > kp.halfL[0]) dx = (me.x - kp.L[0]) - o.x;
        else if (dx < -kp.halfL[0]) dx = me.x - (o.x - kp.L[0]);
        if (dy > kp.halfL[1]) dy = (me.y - kp.L[1]) - o.y;
        else if (dy < -kp.halfL[1]) dy = me.y - (o.y - kp.L[1]);
        if (DIM == 3) {
            if (dz > kp.halfL[2]) dz = (me.z - kp.L[2]) - o.z;
            else if (dz < -kp.halfL[2]) dz = me.z - (o.z - kp.L[2]);
        }
    }
    r2 = DIM == 3 ? fmaf(dx, dx, fmaf(dy, dy, dz * dz)) : fmaf(dx, dx, dy * dy);
}

// Distance (squared) from a particle at offset f in [0,1] (bin units) of its
// bin to the neighbouring bin at offset o in {-1, 0, +1}, bin side b.
__device__ __forceinline__ float gap2(int o, float f, float b)
{
    const float d = o < 0 ? f * b : (o > 0 ? (1.f - f) * b : 0.f);
    return d * d;
}

// Evaluates the listed neighbours of every lane (lanes with an empty list
// idle) and adds them to F. All lanes of the warp call it.
template <int DIM, bool PERIODIC>
__device__ __forceinline__ void flush_list(const KP &kp, const SmemTables &t, const uint32_t *lst, int nl, float4 me,
                                           int row, FAcc &F)
{
    const int m = __reduce_max_sync(0xffffffffu, nl);
    int ax = 0, ay = 0, az = 0;
    for (int i = 0; i < m; ++i) {
        if (i < nl) {
            const float4 o = __ldg(&kp.S[lst[i * 32]]);
            float dx, dy, dz, r2;
            pair_delta<DIM, PERIODIC>(kp, me, o, dx, dy, dz, r2);
            const int st = row + (int)(__float_as_uint(o.w) >> SP_SHIFT);
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            const float f = t.amp_f[st] * (__expf(-r * t.inv_eps[st]) - t.shift[st]);
            const float sq = (f * rinv) * kp.fq_inv;
            ax += __float2int_rn(sq * dx);
            ay += __float2int_rn(sq * dy);
            if (DIM == 3) az += __float2int_rn(sq * dz);
        }
    }
    F.x += ax;
    F.y += ay;
    F.z += az;
}

// Pair force of the particle `me` (sorted index `self`) of every valid lane.
// Must be called by all 32 lanes of the warp (`valid` false for padding lanes).
template <int DIM, bool PERIODIC, bool STATS>
__device__ __forceinline__ float3 pair_force(const KP &kp, const SmemTables &t, uint32_t self, float4 me, int sp,
                                             bool valid, int &count, unsigned long long &idsum, unsigned char *wbuf)
{
    // the warp's region: staged ranges [RowCap][32], then lists [LIST_CAP][32]
    const int lane = threadIdx.x & 31;
    uint2 *rng = reinterpret_cast<uint2 *>(wbuf) + lane;
    uint32_t *lst = reinterpret_cast<uint32_t *>(wbuf + (size_t)32 * RowCap<DIM, PERIODIC>::value * sizeof(uint2)) + lane;
    int c[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f};
    const float pc[3] = {me.x, me.y, me.z};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        c[a] = bin_axis(pc[a], kp.lo[a], kp.inv_b[a], kp.nb[a]);
        f[a] = fminf(fmaxf(__fmul_rn(__fsub_rn(pc[a], kp.lo[a]), kp.inv_b[a]) - (float)c[a], 0.f), 1.f);
        if (kp.search == 2) {
            lo[a] = f[a] < 0.5f ? c[a] - 1 : c[a];
            hi[a] = lo[a] + 1;
        } else {
            lo[a] = c[a] - 1;
            hi[a] = c[a] + 1;
        }
        if (!PERIODIC) {
            lo[a] = max(lo[a], 0);
            hi[a] = min(hi[a], kp.nb[a] - 1);
        }
    }
    if (DIM == 2) c[2] = lo[2] = hi[2] = layer_of(kp, me);  // rows of the particle's own layer
    const float rs2 = kp.rsp2[sp];
    const uint32_t *__restrict__ cnt = kp.cnt_cur;
    const uint32_t *__restrict__ gst = kp.gstart;
    const uint32_t n = (uint32_t)kp.n;
    int nr = 0;
    if (valid) {
        for (int z = lo[2]; z <= hi[2]; ++z) {
            const float gz = DIM == 3 ? gap2(z - c[2], f[2], kp.bside[2]) : 0.f;
            int zz = z;
            if (PERIODIC && DIM == 3) zz = z < 0 ? z + kp.nb[2] : (z >= kp.nb[2] ? z - kp.nb[2] : z);
            for (int y = lo[1]; y <= hi[1]; ++y) {
                const float gyz = gz + gap2(y - c[1], f[1], kp.bside[1]);
                if (gyz >= rs2) continue;  // the whole row is out of reach
                int yy = y;
                if (PERIODIC) yy = y < 0 ? y + kp.nb[1] : (y >= kp.nb[1] ? y - kp.nb[1] : y);
                const uint32_t rowk = (uint32_t)kp.px * ((uint32_t)yy + (uint32_t)kp.nb[1] * (uint32_t)zz);
                int x0 = lo[0], x1 = hi[0];
                if (x0 < c[0] && gyz + gap2(-1, f[0], kp.bside[0]) >= rs2) x0 = c[0];
                if (x1 > c[0] && gyz + gap2(1, f[0], kp.bside[0]) >= rs2) x1 = c[0];
                if (PERIODIC && x0 < 0) {
                    const uint32_t kk = rowk + (uint32_t)(kp.nb[0] - 1);
                    rng[nr++ * 32] = make_uint2(bin_start(cnt, gst, kk), bin_start(cnt, gst, kk + 1));
                    x0 = 0;
                }
                if (PERIODIC && x1 >= kp.nb[0]) {
                    rng[nr++ * 32] = make_uint2(bin_start(cnt, gst, rowk), bin_start(cnt, gst, rowk + 1));
                    x1 = kp.nb[0] - 1;
                }
                if (x0 <= x1)
                    rng[nr++ * 32] = make_uint2(bin_start(cnt, gst, rowk + x0), bin_start(cnt, gst, rowk + x1 + 1));
            }
        }
    }
    const float4 *__restrict__ S = kp.S;
    const int row = sp * MAXS;
    // squared cutoffs against species 0 and 1 in registers (systems of up to
    // two species, the model of the paper); more species read the table
    const bool two = kp.ns <= 2;
    const float rc2_0 = t.rc2[row], rc2_1 = t.rc2[row + 1];
    FAcc F = {0ll, 0ll, 0ll};
    int nl = 0;
    int r = 0;
    uint32_t q = 0, qe = 0;
    while (q >= qe && r < nr) {
        const uint2 g = rng[r++ * 32];
        q = g.x;
        qe = min(g.y, n);  // offsets are trusted only up to n
    }
    bool more = q < qe;
    while (__any_sync(0xffffffffu, more)) {
#if CHEMO_BATCH_LOADS
        // a chunk of up to UNROLL candidates from one range, all loaded
        // before any is tested; past the end of its range a lane tests a
        // far-away sentinel (no pair), so the chunk ends at the warp's longest
        {
            const uint32_t m = more ? min((uint32_t)UNROLL, qe - q) : 0u;
            const uint32_t mw = __reduce_max_sync(0xffffffffu, m);
            float4 ob[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
                ob[u] = (uint32_t)u < m ? __ldg(&S[q + u]) : make_float4(1e30f, 1e30f, 1e30f, 0.f);
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if ((uint32_t)u >= mw) break;
                const float4 o = ob[u];
                const uint32_t qq = q + (uint32_t)u;
                float dx, dy, dz, r2;
                pair_delta<DIM, PERIODIC>(kp, me, o, dx, dy, dz, r2);
                const uint32_t so = __float_as_uint(o.w) >> SP_SHIFT;
                const float rc2 = two ? (so ? rc2_1 : rc2_0) : t.rc2[row + (int)so];
                if (r2 < rc2 && r2 > 0.f && qq != self) {
                    lst[nl++ * 32] = qq;
                    count += 1;
                    if (STATS) idsum += (unsigned long long)(__float_as_uint(o.w) & ID_MASK);
                }
            }
        }
        if (more) {
            const uint32_t m = min((uint32_t)UNROLL, qe - q);
#else
        if (more) {
            const uint32_t m = min((uint32_t)UNROLL, qe - q);
            // a chunk of up to UNROLL candidates from one range; the next
            // candidate is loaded while the current one is tested
            float4 o = __ldg(&S[q]);
            for (uint32_t u = 0; u < m; ++u) {
                const uint32_t qq = q + u;
                const float4 on = u + 1 < m ? __ldg(&S[qq + 1]) : o;
                float dx, dy, dz, r2;
                pair_delta<DIM, PERIODIC>(kp, me, o, dx, dy, dz, r2);
                const uint32_t so = __float_as_uint(o.w) >> SP_SHIFT;
                const float rc2 = two ? (so ? rc2_1 : rc2_0) : t.rc2[row + (int)so];
                if (r2 < rc2 && r2 > 0.f && qq != self) {
                    lst[nl++ * 32] = qq;
                    count += 1;
                    if (STATS) idsum += (unsigned long long)(__float_as_uint(o.w) & ID_MASK);
                }
                o = on;
            }
#endif
            q += m;
            if (q >= qe) {
                while (q >= qe && r < nr) {
                    const uint2 g = rng[r++ * 32];
                    q = g.x;
                    qe = min(g.y, n);
                }
                more = q < qe;
            }
        }
        if (__any_sync(0xffffffffu, nl > LIST_CAP - UNROLL)) {
            flush_list<DIM, PERIODIC>(kp, t, lst, nl, me, row, F);
            nl = 0;
        }
    }
    flush_list<DIM, PERIODIC>(kp, t, lst, nl, me, row, F);
    return make_float3(__ll2float_rn(F.x) * kp.fq, __ll2float_rn(F.y) * kp.fq,
                       DIM == 3 ? __ll2float_rn(F.z) * kp.fq : 0.f);
}

// ---------------------------------------------------------------------------
// Warp-cooperative search (3^d window). The 32 lanes of a warp hold 32
// consecutive cells of the sorted array, so they fall into a few runs of
// cells that share a bin. For each run the warp walks the run's window once:
// the window's candidates are split across the lanes (one coalesced load per
// candidate), and each lane tests its candidate against every cell of the
// run, whose positions are broadcast from shared memory. Pairs inside the
// cutoff go to a queue of the warp (ballot + popc); the queue is evaluated
// in a converged loop, each term added to its cell with a 32-bit shared
// atomic (at most QCAP terms of magnitude < 2^25 per flush, no overflow) and
// drained into 64-bit registers after every flush. The sum is exact, so the
// force is the same as the per-lane search's and independent of the order.
// ---------------------------------------------------------------------------
constexpr int QCAP = 64;  // queue entries; flushed once more than QCAP - 32 are held

template <int DIM, bool PERIODIC>
struct WinRows {
    static constexpr int value = (DIM == 3 ? 9 : 3) * (PERIODIC ? 2 : 1);
};

struct WarpSmem {
    float4 ipos[32];               // the warp's cells: position and species (as a float)
    uint2 queue[QCAP];             // (sorted index of the candidate, lane of the cell)
    int facc[3][32];               // fixed-point force of each cell since the last drain
    int cnt[32];                   // in-cutoff neighbours (stage statistics)
    unsigned long long ids[32];    // sum of neighbour ids (stage statistics)
    uint2 rows[18];                // window ranges of the current run: (first index, first candidate)
};

template <int DIM, bool PERIODIC, bool STATS>
__device__ __forceinline__ void flush_queue(const KP &kp, const SmemTables &t, WarpSmem &ws, int qn, int lane,
                                            long long &Fx, long long &Fy, long long &Fz)
{
    __syncwarp();
    for (int e = lane; e < qn; e += 32) {
        const uint2 ent = ws.queue[e];
        const float4 o = __ldg(&kp.S[ent.x]);
        const float4 pi = ws.ipos[ent.y];
        float dx, dy, dz, r2;
        pair_delta<DIM, PERIODIC>(kp, pi, o, dx, dy, dz, r2);
        if (!(r2 > 0.f)) continue;  // coincident distinct cells exert no force
        const int st = (int)pi.w * MAXS + (int)(__float_as_uint(o.w) >> SP_SHIFT);
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float f = t.amp_f[st] * (__expf(-r * t.inv_eps[st]) - t.shift[st]);
        const float sq = (f * rinv) * kp.fq_inv;
        atomicAdd(&ws.facc[0][ent.y], __float2int_rn(sq * dx));
        atomicAdd(&ws.facc[1][ent.y], __float2int_rn(sq * dy));
        if (DIM == 3) atomicAdd(&ws.facc[2][ent.y], __float2int_rn(sq * dz));
        if (STATS) {
            atomicAdd(&ws.cnt[ent.y], 1);
            atomicAdd(&ws.ids[ent.y], (unsigned long long)(__float_as_uint(o.w) & ID_MASK));
        }
    }
    __syncwarp();
    Fx += ws.facc[0][lane];
    Fy += ws.facc[1][lane];
    Fz += ws.facc[2][lane];
    ws.facc[0][lane] = 0;
    ws.facc[1][lane] = 0;
    ws.facc[2][lane] = 0;
    __syncwarp();
}

// Tests candidate o (squared cutoffs c0 + w c1 against a cell of species
// flag w) against the cells [h, e) of the run: bit k-h set when in reach.
template <int DIM, bool PERIODIC>
__device__ __forceinline__ void test_run2(const KP &kp, const WarpSmem &ws, int h, int e, float4 o0, float a0,
                                          float b0, float4 o1, float a1, float b1, uint32_t &m0, uint32_t &m1)
{
    uint32_t bit = 1u;
#pragma unroll 4
    for (int k = h; k < e; ++k) {
        const float4 pi = ws.ipos[k];
        float dx, dy, dz, r2;
        pair_delta<DIM, PERIODIC>(kp, pi, o0, dx, dy, dz, r2);
        if (r2 < fmaf(pi.w, b0, a0)) m0 |= bit;
        pair_delta<DIM, PERIODIC>(kp, pi, o1, dx, dy, dz, r2);
        if (r2 < fmaf(pi.w, b1, a1)) m1 |= bit;
        bit <<= 1;
    }
}

// Pair force of the cell of every lane; `self` is the lane's sorted index
// (lanes hold consecutive indices). All 32 lanes must call it. A warp whose
// cells fall in more than kp.warp_runs bins (sparse regions, where a run
// holds one or two cells) takes the per-lane search instead.
template <int DIM, bool PERIODIC, bool STATS>
__device__ __forceinline__ float3 pair_force_warp(const KP &kp, const SmemTables &t, unsigned char *wbuf,
                                                  uint32_t self, float4 me, int sp, bool valid, int &count,
                                                  unsigned long long &idsum)
{
    constexpr int NR = WinRows<DIM, PERIODIC>::value;
    const int lane = threadIdx.x & 31;
    const uint32_t base = self - (uint32_t)lane;
    const uint32_t n = (uint32_t)kp.n;
    const int cx = bin_axis(me.x, kp.lo[0], kp.inv_b[0], kp.nb[0]);
    const int cy = bin_axis(me.y, kp.lo[1], kp.inv_b[1], kp.nb[1]);
    const int cz = DIM == 3 ? bin_axis(me.z, kp.lo[2], kp.inv_b[2], kp.nb[2]) : layer_of(kp, me);
    const uint32_t key = valid ? bin_key(kp, cx, cy, cz) : 0xFFFFFFFFu;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    unsigned heads = __ballot_sync(0xffffffffu, valid && (lane == 0 || key != prev));
    if (__popc(heads) > kp.warp_runs) return pair_force<DIM, PERIODIC, STATS>(kp, t, self, me, sp, valid, count, idsum, wbuf);

    WarpSmem &ws = *reinterpret_cast<WarpSmem *>(wbuf);
    ws.ipos[lane] = make_float4(me.x, me.y, me.z, (float)sp);
    ws.facc[0][lane] = 0;
    ws.facc[1][lane] = 0;
    ws.facc[2][lane] = 0;
    if (STATS) {
        ws.cnt[lane] = 0;
        ws.ids[lane] = 0ull;
    }
    const int nvalid = __popc(vmask);  // valid lanes are a prefix of the warp
    const bool two = kp.ns <= 2;
    const uint32_t *__restrict__ cnt = kp.cnt_cur;
    const uint32_t *__restrict__ gst = kp.gstart;
    const unsigned lt = (1u << lane) - 1u;
    long long Fx = 0, Fy = 0, Fz = 0;
    int qn = 0, npairs = 0;
    __syncwarp();
    while (heads) {
        const int h = __ffs(heads) - 1;
        heads &= heads - 1u;
        const int e = heads ? __ffs(heads) - 1 : nvalid;  // the run is lanes [h, e)
        const int bx = __shfl_sync(0xffffffffu, cx, h);
        const int by = __shfl_sync(0xffffffffu, cy, h);
        const int bz = __shfl_sync(0xffffffffu, cz, h);
        // window ranges: lane r < NR owns range r (row, and for a periodic
        // row the wrapped end bin as a second piece)
        uint32_t q0 = 0, q1 = 0;
        if (lane < NR) {
            const int piece = PERIODIC ? lane / (NR / 2) : 0;
            const int rr = PERIODIC ? lane % (NR / 2) : lane;
            const int dy = (DIM == 3 ? rr % 3 : rr) - 1;
            const int dz = DIM == 3 ? rr / 3 - 1 : 0;
            int y = by + dy, z = bz + dz;
            bool ok = true;
            if (PERIODIC) {
                y = y < 0 ? y + kp.nb[1] : (y >= kp.nb[1] ? y - kp.nb[1] : y);
                if (DIM == 3) z = z < 0 ? z + kp.nb[2] : (z >= kp.nb[2] ? z - kp.nb[2] : z);
            } else {
                ok = y >= 0 && y < kp.nb[1] && (DIM == 2 || (z >= 0 && z < kp.nb[2]));
            }
            int x0 = bx - 1, x1 = bx + 1;
            if (PERIODIC) {
                if (piece == 0) {
                    x0 = max(x0, 0);
                    x1 = min(x1, kp.nb[0] - 1);
                } else if (bx - 1 < 0) {
                    x0 = x1 = kp.nb[0] - 1;
                } else if (bx + 1 >= kp.nb[0]) {
                    x0 = x1 = 0;
                } else {
                    ok = false;
                }
            } else {
                x0 = max(x0, 0);
                x1 = min(x1, kp.nb[0] - 1);
            }
            if (ok) {
                const uint32_t rowk = (uint32_t)kp.px * ((uint32_t)y + (uint32_t)kp.nb[1] * (uint32_t)z);
                q0 = min(bin_start(cnt, gst, rowk + (uint32_t)x0), n);
                q1 = min(bin_start(cnt, gst, rowk + (uint32_t)x1 + 1u), n);
                q1 = max(q1, q0);
            }
        }
        const uint32_t len = q1 - q0;
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (lane < NR) ws.rows[lane] = make_uint2(q0, incl - len);
        __syncwarp();
        // candidate passes of 64: lane takes candidates t0 + lane and
        // t0 + 32 + lane and tests both against every cell of the run (bit
        // masks of hits); the hits then go to the queue in ballot rounds
        int r = 0;
        const uint32_t first = base + (uint32_t)h;
        const uint32_t runlen = (uint32_t)(e - h);
        for (uint32_t t0 = 0; t0 < total; t0 += 64) {
            uint32_t qa = 0xFFFFFFFFu, qb = 0xFFFFFFFFu;
            float4 oa = make_float4(0.f, 0.f, 0.f, 0.f), ob = oa;
            const uint32_t ta = t0 + (uint32_t)lane, tb = ta + 32u;
            if (ta < total) {
                while (r + 1 < NR && ws.rows[r + 1].y <= ta) ++r;
                qa = ws.rows[r].x + (ta - ws.rows[r].y);
                oa = __ldg(&kp.S[qa]);
            }
            if (tb < total) {
                while (r + 1 < NR && ws.rows[r + 1].y <= tb) ++r;
                qb = ws.rows[r].x + (tb - ws.rows[r].y);
                ob = __ldg(&kp.S[qb]);
            }
            // squared cutoffs against species 0 (a) and the step to species 1 (b);
            // no candidate: negative, never in reach
            float aa = -1.f, ba = 0.f, ab = -1.f, bb = 0.f;
            uint32_t ma = 0u, mb = 0u;
            const uint32_t sa = __float_as_uint(oa.w) >> SP_SHIFT, sb = __float_as_uint(ob.w) >> SP_SHIFT;
            if (two) {
                if (qa != 0xFFFFFFFFu) {
                    aa = t.rc2[sa];
                    ba = t.rc2[MAXS + sa] - aa;
                }
                if (qb != 0xFFFFFFFFu) {
                    ab = t.rc2[sb];
                    bb = t.rc2[MAXS + sb] - ab;
                }
                test_run2<DIM, PERIODIC>(kp, ws, h, e, oa, aa, ba, ob, ab, bb, ma, mb);
            } else {
                uint32_t bit = 1u;
                for (int k = h; k < e; ++k) {
                    const float4 pi = ws.ipos[k];
                    const int row = (int)pi.w * MAXS;
                    float dx, dy, dz, r2;
                    pair_delta<DIM, PERIODIC>(kp, pi, oa, dx, dy, dz, r2);
                    if (qa != 0xFFFFFFFFu && r2 < t.rc2[row + (int)sa]) ma |= bit;
                    pair_delta<DIM, PERIODIC>(kp, pi, ob, dx, dy, dz, r2);
                    if (qb != 0xFFFFFFFFu && r2 < t.rc2[row + (int)sb]) mb |= bit;
                    bit <<= 1;
                }
            }
            if (qa - first < runlen) ma &= ~(1u << (qa - first));  // j != i
            if (qb - first < runlen) mb &= ~(1u << (qb - first));
            while (__any_sync(0xffffffffu, (ma | mb) != 0u)) {
                const bool hb = (ma | mb) != 0u;
                const unsigned hm = __ballot_sync(0xffffffffu, hb);
                if (hb) {
                    uint32_t q;
                    int k;
                    if (ma) {
                        k = h + __ffs(ma) - 1;
                        ma &= ma - 1u;
                        q = qa;
                    } else {
                        k = h + __ffs(mb) - 1;
                        mb &= mb - 1u;
                        q = qb;
                    }
                    ws.queue[qn + __popc(hm & lt)] = make_uint2(q, (uint32_t)k);
                }
                qn += __popc(hm);
                npairs += __popc(hm);
                if (qn > QCAP - 32) {
                    flush_queue<DIM, PERIODIC, STATS>(kp, t, ws, qn, lane, Fx, Fy, Fz);
                    qn = 0;
                }
            }
        }
        __syncwarp();
    }
    flush_queue<DIM, PERIODIC, STATS>(kp, t, ws, qn, lane, Fx, Fy, Fz);
    if (STATS) {
        count += ws.cnt[lane];
        idsum += ws.ids[lane];
    } else if (lane == 0) {
        count += npairs;  // the warp's pairs (profiling; coincident cells included)
    }
    return make_float3(__ll2float_rn(Fx) * kp.fq, __ll2float_rn(Fy) * kp.fq, DIM == 3 ? __ll2float_rn(Fz) * kp.fq : 0.f);
}

// Shared memory of one warp of a pair kernel: the per-lane search stages
// [RowCap][32] ranges and [LIST_CAP][32] list entries; the warp search uses a
// WarpSmem (the hybrid kernel reserves the larger of the two).
template <int DIM, bool PERIODIC, bool WARP>
constexpr size_t warp_region()
{
    constexpr size_t lane_bytes = (size_t)32 * RowCap<DIM, PERIODIC>::value * sizeof(uint2) +
                                  (size_t)32 * LIST_CAP * sizeof(uint32_t);
    constexpr size_t r = WARP && sizeof(WarpSmem) > lane_bytes ? sizeof(WarpSmem) : lane_bytes;
    return (r + 15) & ~(size_t)15;
}

// Dynamic shared memory of the kernels that evaluate pair forces: species
// tables and one region per warp.
template <int DIM, bool PERIODIC, bool WARP, int BT = TPB>
constexpr size_t pair_smem()
{
    return sizeof(SmemTables) + (size_t)(BT / 32) * warp_region<DIM, PERIODIC, WARP>();
}

// ---------------------------------------------------------------------------
// Gradient of c interpolated to a point (Sect. 3.5 D1x/D1y central
// differences at the nodes, mirror ghosts at walls, then multilinear
// interpolation, Sect. 3.6). Also returns the interpolated c.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Half-window search (search mode 4). Every unordered pair is found once, by
// the cell whose window holds the other in its upper half: the rows at
// (dz, dy) > (0, 0) in lexicographic order with all their bins, and in its own
// row the next bin and the cells of its own bin that follow it in the sorted
// array (3D: 4 rows and a part of the own row, against 9 rows; 2D: 1 row and a
// part, against 3). Each term is added to the finder and, negated, to the
// partner with a 64-bit integer atomic. The quantised term is odd in the
// difference vector (negated differences give the same distance, and
// round-to-nearest-even is odd), and integer sums do not depend on the order
// of the additions, so each cell's force is the full window's bit for bit.
// Needs at least 3 bins on a periodic axis (then the 3^d offsets are distinct
// bins and each pair of bins is visited from one side only).
// ---------------------------------------------------------------------------
template <int DIM, bool PERIODIC>
__device__ __forceinline__ void flush_half(const KP &kp, const SmemTables &t, const uint32_t *lst, int nl, float4 me,
                                           int row, FAcc &F)
{
    constexpr int FS = FhStride<DIM>::value;
    const int m = __reduce_max_sync(0xffffffffu, nl);
    int ax = 0, ay = 0, az = 0;
    for (int i = 0; i < m; ++i) {
        if (i < nl) {
            const uint32_t qq = lst[i * 32];
            const float4 o = __ldg(&kp.S[qq]);
            float dx, dy, dz, r2;
            pair_delta<DIM, PERIODIC>(kp, me, o, dx, dy, dz, r2);
            const int st = row + (int)(__float_as_uint(o.w) >> SP_SHIFT);
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            const float f = t.amp_f[st] * (__expf(-r * t.inv_eps[st]) - t.shift[st]);
            const float sq = (f * rinv) * kp.fq_inv;
            const int tx = __float2int_rn(sq * dx), ty = __float2int_rn(sq * dy);
            ax += tx;
            ay += ty;
            unsigned long long *pf = reinterpret_cast<unsigned long long *>(kp.Fh) + (size_t)qq * FS;
            atomicAdd(pf + 0, (unsigned long long)(long long)(-tx));
            atomicAdd(pf + 1, (unsigned long long)(long long)(-ty));
            if (DIM == 3) {
                const int tz = __float2int_rn(sq * dz);
                az += tz;
                atomicAdd(pf + 2, (unsigned long long)(long long)(-tz));
            }
        }
    }
    F.x += ax;
    F.y += ay;
    F.z += az;
}

// Ranges of the upper half of the 3^d window of the cell `me` (sorted index
// j): the rows at (dz, dy) > (0, 0) in lexicographic order with all their
// bins, in its own row the next bin and the cells of its own bin after it.
// Calls push(first, end) for each range of sorted indices.
template <int DIM, bool PERIODIC, typename Push>
__device__ __forceinline__ void stage_half(const KP &kp, float4 me, int sp, uint32_t j, Push &&push)
{
    const uint32_t *__restrict__ cnt = kp.cnt_cur;
    const uint32_t *__restrict__ gst = kp.gstart;
    const float rs2 = kp.rsp2[sp];
    int c[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f};
    const float pc[3] = {me.x, me.y, me.z};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        c[a] = bin_axis(pc[a], kp.lo[a], kp.inv_b[a], kp.nb[a]);
        f[a] = fminf(fmaxf(__fmul_rn(__fsub_rn(pc[a], kp.lo[a]), kp.inv_b[a]) - (float)c[a], 0.f), 1.f);
    }
    if (DIM == 2) c[2] = layer_of(kp, me);  // rows of the particle's own layer
    // rows (oy, oz) of the upper half: the own row (0, 0), then (1, 0),
    // then (-1..1, 1) in 3D
    constexpr int NROWS = DIM == 3 ? 5 : 2;
    for (int k = 0; k < NROWS; ++k) {
        const int oy = k == 0 ? 0 : (k == 1 ? 1 : k - 3);
        const int oz = k < 2 ? 0 : 1;
        int y = c[1] + oy, z = c[2] + oz;
        if (PERIODIC) {
            y = y < 0 ? y + kp.nb[1] : (y >= kp.nb[1] ? y - kp.nb[1] : y);
            if (DIM == 3) z = z >= kp.nb[2] ? z - kp.nb[2] : z;
        } else if (y < 0 || y >= kp.nb[1] || (DIM == 3 && z >= kp.nb[2])) {
            continue;
        }
        const float gyz = (DIM == 3 ? gap2(oz, f[2], kp.bside[2]) : 0.f) + gap2(oy, f[1], kp.bside[1]);
        if (gyz >= rs2) continue;  // the whole row is out of reach
        const uint32_t rowk = (uint32_t)kp.px * ((uint32_t)y + (uint32_t)kp.nb[1] * (uint32_t)z);
        int x0 = k == 0 ? c[0] : c[0] - 1, x1 = c[0] + 1;
        if (!PERIODIC) {
            x0 = max(x0, 0);
            x1 = min(x1, kp.nb[0] - 1);
        }
        if (x0 < c[0] && gyz + gap2(-1, f[0], kp.bside[0]) >= rs2) x0 = c[0];
        if (x1 > c[0] && gyz + gap2(1, f[0], kp.bside[0]) >= rs2) x1 = c[0];
        if (PERIODIC && x0 < 0) {
            const uint32_t kk = rowk + (uint32_t)(kp.nb[0] - 1);
            push(bin_start(cnt, gst, kk), bin_start(cnt, gst, kk + 1));
            x0 = 0;
        }
        if (PERIODIC && x1 >= kp.nb[0]) {
            push(bin_start(cnt, gst, rowk), bin_start(cnt, gst, rowk + 1));
            x1 = kp.nb[0] - 1;
        }
        if (x0 <= x1) {
            // the own row starts after this cell: the cells of its bin
            // before it found the pair themselves
            const uint32_t b0 = k == 0 ? j + 1u : bin_start(cnt, gst, rowk + x0);
            push(b0, bin_start(cnt, gst, rowk + x1 + 1));
        }
    }
}

// BT threads per block; resident blocks per SM scale so that every block
// size keeps the same register budget per thread.
template <int DIM, bool PERIODIC, int BT = TPB>
__global__ void __launch_bounds__(BT, CHEMO_PAIR_BLOCKS *TPB / BT) k_pairs_half(KP kp)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemTables &t = *reinterpret_cast<SmemTables *>(smem);
    load_tables(kp, t);
    __syncthreads();
    constexpr int FS = FhStride<DIM>::value;
    const int64_t j = (int64_t)blockIdx.x * BT + threadIdx.x;
    const bool valid = j < kp.n;
    const float4 me = valid ? kp.S[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int sp = (int)(__float_as_uint(me.w) >> SP_SHIFT);
    const int lane = threadIdx.x & 31;
    unsigned char *wbuf = smem + sizeof(SmemTables) + (threadIdx.x >> 5) * warp_region<DIM, PERIODIC, false>();
    uint2 *rng = reinterpret_cast<uint2 *>(wbuf) + lane;
    uint32_t *lst = reinterpret_cast<uint32_t *>(wbuf + (size_t)32 * RowCap<DIM, PERIODIC>::value * sizeof(uint2)) + lane;
    const uint32_t n = (uint32_t)kp.n;
    int nr = 0;
    if (valid) stage_half<DIM, PERIODIC>(kp, me, sp, (uint32_t)j, [&](uint32_t x0, uint32_t x1) {
        rng[nr++ * 32] = make_uint2(x0, x1);
    });
    const float4 *__restrict__ S = kp.S;
    const int row = sp * MAXS;
    const bool two = kp.ns <= 2;
    const float rc2_0 = t.rc2[row], rc2_1 = t.rc2[row + 1];
    FAcc F = {0ll, 0ll, 0ll};
    int count = 0, nl = 0, r = 0;
    uint32_t tests = 0;  // candidates tested (profiling)
    uint32_t q = 0, qe = 0;
    while (q >= qe && r < nr) {
        const uint2 g = rng[r++ * 32];
        q = g.x;
        qe = min(g.y, n);  // offsets are trusted only up to n
    }
    bool more = q < qe;
    while (__any_sync(0xffffffffu, more)) {
        // a chunk of up to UNROLL candidates per lane, all loaded before any
        // is tested; past the end of its range a lane tests a far-away
        // sentinel (no pair), so the chunk ends at the warp's longest
        // (a branch the whole warp takes together)
        const uint32_t m = more ? min((uint32_t)UNROLL, qe - q) : 0u;
        tests += m;
        const uint32_t mw = __reduce_max_sync(0xffffffffu, m);
        float4 ob[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            ob[u] = (uint32_t)u < m ? __ldg(&S[q + u]) : make_float4(1e30f, 1e30f, 1e30f, 0.f);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            if ((uint32_t)u >= mw) break;
            const float4 o = ob[u];
            float dx, dy, dz, r2;
            pair_delta<DIM, PERIODIC>(kp, me, o, dx, dy, dz, r2);
            const uint32_t so = __float_as_uint(o.w) >> SP_SHIFT;
            const float rc2 = two ? (so ? rc2_1 : rc2_0) : t.rc2[row + (int)so];
            if (r2 < rc2 && r2 > 0.f) lst[nl++ * 32] = q + (uint32_t)u;
        }
        if (more) {
            q += m;
            if (q >= qe) {
                while (q >= qe && r < nr) {
                    const uint2 g = rng[r++ * 32];
                    q = g.x;
                    qe = min(g.y, n);
                }
                more = q < qe;
            }
        }
        if (__any_sync(0xffffffffu, nl > LIST_CAP - UNROLL)) {
            flush_half<DIM, PERIODIC>(kp, t, lst, nl, me, row, F);
            count += nl;
            nl = 0;
        }
    }
    flush_half<DIM, PERIODIC>(kp, t, lst, nl, me, row, F);
    count += nl;
    if (kp.pair_count) {  // profiling only: each pair found here is an in-cutoff pair of both cells
        const int wsum = __reduce_add_sync(0xffffffffu, count);
        if (lane == 0 && wsum) atomicAdd(kp.pair_count + (blockIdx.x & (PROF_SLOTS - 1)), 2ull * (unsigned long long)wsum);
    }
    if (kp.test_count) {  // profiling only: candidates tested
        const uint32_t tsum = __reduce_add_sync(0xffffffffu, tests);
        if (lane == 0 && tsum) atomicAdd(kp.test_count + (blockIdx.x & (PROF_SLOTS - 1)), (unsigned long long)tsum);
    }
    if (valid && (F.x | F.y | F.z)) {
        unsigned long long *pf = reinterpret_cast<unsigned long long *>(kp.Fh) + (size_t)j * FS;
        atomicAdd(pf + 0, (unsigned long long)F.x);
        atomicAdd(pf + 1, (unsigned long long)F.y);
        if (DIM == 3) atomicAdd(pf + 2, (unsigned long long)F.z);
    }
}

// Offsets from the base node are taken in IT (32-bit for grids of fewer than
// 2^31 nodes: one address multiply-add per load instead of 64-bit adds).
template <int DIM, typename IT>
__device__ __forceinline__ float3 grad_interp_t(const KP &kp, const float *__restrict__ c, float4 p, float &cval)
{
    int i0, i1, j0, j1, k0 = 0, k1 = 0;
    float fx, fy, fz = 0.f;
    gcell(kp, 0, p.x, i0, i1, fx);
    gcell(kp, 1, p.y, j0, j1, fy);
    if (DIM == 3) gcell(kp, 2, p.z, k0, k1, fz);
    else k0 = layer_of(kp, p);  // the particle's own layer of the grid
    const IT gx = kp.g[0], plane = (IT)kp.g[0] * (IT)kp.g[1];
    // base node (i0, j0, k0) and offsets to the other nodes used
    c += (int64_t)i0 + (int64_t)kp.g[0] * ((int64_t)j0 + (int64_t)kp.g[1] * k0);
    const IT b = 0;
    const IT ox[4] = {(IT)(gnbr(kp, 0, i0 - 1) - i0), 0, (IT)(i1 - i0), (IT)(gnbr(kp, 0, i1 + 1) - i0)};
    const IT oy[4] = {(IT)(gnbr(kp, 1, j0 - 1) - j0) * gx, 0, (IT)(j1 - j0) * gx, (IT)(gnbr(kp, 1, j1 + 1) - j0) * gx};
    IT oz[4] = {0, 0, 0, 0};
    if (DIM == 3) {
        oz[0] = (IT)(gnbr(kp, 2, k0 - 1) - k0) * plane;
        oz[2] = (IT)(k1 - k0) * plane;
        oz[3] = (IT)(gnbr(kp, 2, k1 + 1) - k0) * plane;
    }
    constexpr int NZ = DIM == 3 ? 2 : 1;
    // corners C[bz][by][bx] and the nodes one beyond them along each axis
    float C[NZ][2][2], XM[NZ][2], XP[NZ][2], YM[NZ][2], YP[NZ][2], ZM[2][2], ZP[2][2];
#pragma unroll
    for (int bz = 0; bz < NZ; ++bz) {
        const IT z = oz[1 + bz];  // plane k0 (offset 0) or k1
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const IT yb = oy[1 + bb], xb = ox[1 + bb];
            C[bz][bb][0] = __ldg(&c[b + z + yb]);
            C[bz][bb][1] = __ldg(&c[b + z + yb + ox[2]]);
            XM[bz][bb] = __ldg(&c[b + z + yb + ox[0]]);
            XP[bz][bb] = __ldg(&c[b + z + yb + ox[3]]);
            YM[bz][bb] = __ldg(&c[b + z + oy[0] + xb]);
            YP[bz][bb] = __ldg(&c[b + z + oy[3] + xb]);
        }
    }
    if (DIM == 3) {
#pragma unroll
        for (int by = 0; by < 2; ++by)
#pragma unroll
            for (int bx = 0; bx < 2; ++bx) {
                ZM[by][bx] = __ldg(&c[b + oz[0] + oy[1 + by] + ox[1 + bx]]);
                ZP[by][bx] = __ldg(&c[b + oz[3] + oy[1 + by] + ox[1 + bx]]);
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
                const float gxv = bx ? XP[bz][by] - C[bz][by][0] : C[bz][by][1] - XM[bz][by];
                const float gyv = by ? YP[bz][bx] - C[bz][0][bx] : C[bz][1][bx] - YM[bz][bx];
                g.x = fmaf(w, gxv, g.x);
                g.y = fmaf(w, gyv, g.y);
                if (DIM == 3) {
                    const float gzv = bz ? ZP[by][bx] - C[0][by][bx] : C[NZ - 1][by][bx] - ZM[by][bx];
                    g.z = fmaf(w, gzv, g.z);
                }
                cval = fmaf(w, C[bz][by][bx], cval);
            }
    g.x *= kp.inv_2h[0];
    g.y *= kp.inv_2h[1];
    g.z *= DIM == 3 ? kp.inv_2h[2] : 0.f;
    return g;
}

template <int DIM>
__device__ __forceinline__ float3 grad_interp(const KP &kp, const float *__restrict__ c, float4 p, float &cval)
{
    return kp.G < ((int64_t)1 << 31) ? grad_interp_t<DIM, int>(kp, c, p, cval)
                                     : grad_interp_t<DIM, int64_t>(kp, c, p, cval);
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
#ifndef CHEMO_MOVE_BLOCKS
#define CHEMO_MOVE_BLOCKS 6
#endif
// HALF: the pair force was summed by the half-window kernel; this instance
// holds no search code (fewer registers, small shared memory, more warps to
// hide the latency of the gathers).
template <int DIM, bool PERIODIC, bool WARP, bool HALF = false, int BT = TPB>
__global__ void __launch_bounds__(BT, (HALF ? CHEMO_MOVE_BLOCKS : CHEMO_PAIR_BLOCKS) * TPB / BT) k_step(KP kp, int cur)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemTables &t = *reinterpret_cast<SmemTables *>(smem);
    if (!HALF) load_tables(kp, t);  // the half-window instance evaluates no pair terms
    const int64_t j = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (kp.zero_src) {  // source grids of the last step, read by its PDE: cleared for this step's deposit
        for (int64_t g = j; g < kp.G; g += (int64_t)gridDim.x * BT) {
            kp.srcg[g] = 0.f;
            kp.Rg[g] = 0.f;
        }
    }
    // adjoint recording: this step's count table, group offsets and field
    unsigned long long tk = kp.tape.pos ? *kp.step - kp.tape.s0 : ~0ull;
    if (kp.tape.pos && kp.tape.period) tk %= kp.tape.period;
    const bool taping = tk < kp.tape.nk;
    if (taping) {
        const int64_t stride = (int64_t)gridDim.x * BT;
        for (int64_t i = j; i < kp.tape.cwords; i += stride) kp.tape.cnt[(int64_t)tk * kp.tape.cwords + i] = kp.cnt_cur[i];
        for (int64_t i = j; i < kp.tape.gwords; i += stride) kp.tape.gst[(int64_t)tk * kp.tape.gwords + i] = kp.gstart[i];
        if (kp.has_grid)
            for (int64_t i = j; i < kp.G; i += stride) kp.tape.c[(int64_t)tk * kp.G + i] = kp.c[cur][i];
    }
    if (!HALF) __syncthreads();
    const bool valid = j < kp.n;
    const float4 me = valid ? kp.S[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t w = __float_as_uint(me.w);
    const uint32_t id = w & ID_MASK;
    const uint32_t layer = (uint32_t)layer_of(kp, me);
    int sp = (int)(w >> SP_SHIFT);

    int npairs = 0;
    unsigned long long ids_unused = 0ull;
    float3 F = make_float3(0.f, 0.f, 0.f);
    if constexpr (HALF) {
        // summed by the half-window kernel (the scatter clears them for the next step)
        if (valid && kp.pairs) {
            constexpr int FS = FhStride<DIM>::value;
            const longlong2 a = reinterpret_cast<const longlong2 *>(kp.Fh + (size_t)j * FS)[0];
            const long long az = DIM == 3 ? kp.Fh[(size_t)j * FS + 2] : 0ll;
            F = make_float3(__ll2float_rn(a.x) * kp.fq, __ll2float_rn(a.y) * kp.fq,
                            DIM == 3 ? __ll2float_rn(az) * kp.fq : 0.f);
        }
    } else {
        if (kp.pairs) {  // warp-synchronous: every lane takes part
            unsigned char *wbuf = smem + sizeof(SmemTables) + (threadIdx.x >> 5) * warp_region<DIM, PERIODIC, WARP>();
            if (WARP)
                F = pair_force_warp<DIM, PERIODIC, false>(kp, t, wbuf, (uint32_t)j, me, sp, valid, npairs, ids_unused);
            else
                F = pair_force<DIM, PERIODIC, false>(kp, t, (uint32_t)j, me, sp, valid, npairs, ids_unused, wbuf);
        }
        if (kp.pair_count) {  // profiling only: in-cutoff pairs of this step
            const int wsum = __reduce_add_sync(0xffffffffu, npairs);
            if ((threadIdx.x & 31) == 0 && wsum)
                atomicAdd(kp.pair_count + (blockIdx.x & (PROF_SLOTS - 1)), (unsigned long long)wsum);
        }
    }
    if (!valid) return;
    if (kp.sub && id == ID_MASK) {  // a ghost stays put: its own sub-domain moves it
        kp.U[j] = me;
        if (kp.dS) kp.dU[j] = kp.dS[j];
        kp.slot[j] = count_bin(kp.cnt_nxt, key_of(kp, me), kp.err);
        return;
    }
    if (taping) {  // recorded for the adjoint: the state before the move and the pair force
        const int64_t gi = gid_of(kp, me);
        const int64_t r = ((int64_t)tk * kp.n + gi) * DIM;
        const int64_t ps = (int64_t)tk + (kp.tape.pos_gap ? (int64_t)(tk / kp.tape.pos_gap) : 0);
        const int64_t rp = (ps * kp.n + gi) * DIM;
        kp.tape.pos[rp + 0] = me.x;
        kp.tape.pos[rp + 1] = me.y;
        if (DIM == 3) kp.tape.pos[rp + 2] = me.z;
        kp.tape.F[r + 0] = F.x;
        kp.tape.F[r + 1] = F.y;
        if (DIM == 3) kp.tape.F[r + 2] = F.z;
        kp.tape.S[(int64_t)tk * kp.n + j] = me;
    }
    const unsigned long long step = *kp.step;

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
    const uint4 rw = cell_words(kp, id, step, TAG_MOVE, layer);
    const float2 n01 = box_muller(rw.x, rw.y);
    float n2 = 0.f;
    if (DIM == 3) n2 = box_muller(rw.z, rw.w).x;
    const float amp = kp.noise[sp];
    // drift increment dt a, or dt a / (1 + dt |a|) for the tamed scheme
    float sc = kp.dt;
    if (kp.move_scheme == 1) {
        const float ax = F.x + dr.x, ay = F.y + dr.y, az = DIM == 3 ? F.z + dr.z : 0.f;
        sc = kp.dt / (1.f + kp.dt * sqrtf(fmaf(ax, ax, fmaf(ay, ay, az * az))));
    }
    const float x1 = me.x + sc * (F.x + dr.x) + amp * n01.x;
    const float y1 = me.y + sc * (F.y + dr.y) + amp * n01.y;
    const float z1 = DIM == 3 ? me.z + sc * (F.z + dr.z) + amp * n2 : 0.f;

    // fixed-step switching (Sect. 3.4): switch when u < rate dt. The
    // comparison that decides the species is taken in double precision, the
    // precision of the paper's code; u = (w + 1/2) 2^-32 is exact there.
    if (kp.reactions) {
        const uint4 rr = cell_words(kp, id, step, TAG_REACT, layer);
        const double u = ((double)rr.x + 0.5) * 2.3283064365386963e-10;
        const double prop = ((double)kp.rk0[sp] + (double)kp.rkc[sp] * (double)conc) * kp.dt_d;
        if (u < prop) sp = kp.rto[sp];
    }

    float xb, yb, zb;
    if (PERIODIC) {
        xb = wrap_axis(x1, kp.lo[0], kp.hi[0], kp.L[0]);
        yb = wrap_axis(y1, kp.lo[1], kp.hi[1], kp.L[1]);
        zb = DIM == 3 ? wrap_axis(z1, kp.lo[2], kp.hi[2], kp.L[2]) : me.z;
    } else {
        xb = reflect_axis(x1, kp.lo[0], kp.hi[0]);
        yb = reflect_axis(y1, kp.lo[1], kp.hi[1]);
        if (DIM == 3 && kp.open_z)  // walls only where the face is the system's
            zb = reflect_axis(z1, (kp.open_z & 1) ? -INFINITY : kp.lo[2], (kp.open_z & 2) ? INFINITY : kp.hi[2]);
        else
            zb = DIM == 3 ? reflect_axis(z1, kp.lo[2], kp.hi[2]) : me.z;
    }
    const bool finite = isfinite(x1) && isfinite(y1) && (DIM == 2 || isfinite(z1));
    if (!finite) {
        set_err(kp, ERR_NONFINITE);
        xb = me.x;
        yb = me.y;
        zb = me.z;
    }
    if (DIM == 3 && kp.open_z && (zb < kp.lo[2] || zb > kp.hi[2])) {  // beyond the halo of an inner face
        set_err(kp, ERR_DOMAIN);
        zb = fminf(fmaxf(zb, kp.lo[2]), kp.hi[2]);
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
    kp.slot[j] = count_bin(kp.cnt_nxt, key_of(kp, nu), kp.err);
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
    // layer of entry i: the last l with layer_off[l] <= i (binary search)
    int64_t local = i;
    if (kp.layers > 1) {
        int l0 = 0, l1 = kp.layers;
        while (l1 - l0 > 1) {
            const int mid = (l0 + l1) >> 1;
            if (kp.layer_off[mid] <= i) l0 = mid;
            else l1 = mid;
        }
        local = i - kp.layer_off[l0];
        x[2] = (float)l0;
    }
    const float4 u = make_float4(x[0], x[1], x[2], __uint_as_float((uint32_t)local | (s << SP_SHIFT)));
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
    kp.slot[i] = count_bin(kp.cnt_nxt, key_of(kp, u), kp.err);
}

// ---------------------------------------------------------------------------
// k_scan: offsets of the groups of 8 bins of the state just counted
// (cnt_nxt): gstart[g] = sum of the counts of all earlier groups,
// gstart[ngroups] = n; each nonempty group's counts are replaced by the
// offsets of its bins within the group. Single pass with decoupled look-back (Merrill &
// Garland, 2016): tiles are claimed in order from an atomic counter, each
// publishes its aggregate, then its inclusive prefix once its predecessors'
// are known. Waits are bounded; a wait that runs out latches ERR_TIMEOUT and
// proceeds. The kernel also clears cnt_cur (the counts of the state the
// particle kernel has finished reading), which the next step counts into.
// ---------------------------------------------------------------------------
#ifndef CHEMO_SCAN_ITEMS
#define CHEMO_SCAN_ITEMS 8
#endif
constexpr int SCAN_ITEMS = CHEMO_SCAN_ITEMS;        // consecutive groups per thread
constexpr int SCAN_TILE = TPB * SCAN_ITEMS;         // groups per tile
// the tile status table is allocated for tiles of at least 2048 groups
static_assert(SCAN_TILE >= 2048, "scan tiles smaller than the tile table allows");
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
    return (wid ? warp_sums[wid - 1] : 0u) + x - v;
}

__device__ __forceinline__ uint32_t halfsum(uint32_t w) { return (w & 0xFFFFu) + (w >> 16); }

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
    const int64_t NG = kp.ngroups;
    const int64_t g0 = (int64_t)tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;

    // group totals of the tile, read (and the other count buffer cleared)
    // with consecutive threads on consecutive groups, then taken back from
    // shared memory as SCAN_ITEMS consecutive groups per thread (one padding
    // word per 32 keeps both passes free of bank conflicts)
    __shared__ uint32_t s_v[SCAN_TILE + SCAN_TILE / 32];
    uint4 *src = reinterpret_cast<uint4 *>(kp.cnt_nxt);  // one uint4 per group
    uint4 *clr = reinterpret_cast<uint4 *>(kp.cnt_cur);
    const int64_t tbase = (int64_t)tile * SCAN_TILE;
    // all of a thread's loads first: the in-place offsets stored below go to
    // the same array, so loads after them could not be issued before them
    // (each thread would wait for one DRAM round trip per group)
    uint4 qv[SCAN_ITEMS];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t g = tbase + i * TPB + (int)threadIdx.x;
        qv[i] = g < NG ? __ldcs(src + g) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int k = i * TPB + (int)threadIdx.x;
        const int64_t g = tbase + k;
        uint32_t s = 0u;
        if (g < NG) {
            const uint4 q = qv[i];
            s = halfsum(q.x) + halfsum(q.y) + halfsum(q.z) + halfsum(q.w);
            clr[g] = make_uint4(0u, 0u, 0u, 0u);
            if (s) {
                // the group's counts become the offsets of its bins within the
                // group (exclusive prefix sums, 16 bits each): a bin's start is
                // then its group's offset plus one 16-bit load (bin_start)
                const uint32_t p1 = q.x & 0xFFFFu, p2 = p1 + (q.x >> 16), p3 = p2 + (q.y & 0xFFFFu);
                const uint32_t p4 = p3 + (q.y >> 16), p5 = p4 + (q.z & 0xFFFFu), p6 = p5 + (q.z >> 16);
                const uint32_t p7 = p6 + (q.w & 0xFFFFu);
                if (p7 > 0xFFFFu) set_err(kp, ERR_OVERFLOW);
                src[g] = make_uint4(p1 << 16, p2 | (p3 << 16), p4 | (p5 << 16), p6 | (p7 << 16));
            }
        }
        s_v[k + (k >> 5)] = s;
    }
    __syncthreads();
    uint32_t v[SCAN_ITEMS];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int k = (int)threadIdx.x * SCAN_ITEMS + i;
        v[i] = s_v[k + (k >> 5)];
    }
    uint32_t tsum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) tsum += v[i];
    uint32_t tile_total;
    const uint32_t tpre = block_exscan(tsum, tile_total, s_warp);

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
                uint32_t spins = 0;
                for (;;) {
                    stw = *(volatile unsigned long long *)&kp.tiles[p];
                    const uint32_t e = (uint32_t)(stw >> 40);
                    flag = (stw >> ST_VAL_BITS) & 3ull;
                    if (e == epoch && flag != 0ull) break;
                    if (++spins > kp.scan_spins) {  // bounded wait
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
            if (tile != 0) atomicExch(&kp.tiles[tile], st_pack(epoch, ST_INC, excl + tile_total));
            s_prefix = excl;
        }
    }
    __syncthreads();
    uint32_t run = (uint32_t)s_prefix + tpre;
    uint32_t out[SCAN_ITEMS];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        out[i] = run;
        run += v[i];
    }
    if (g0 + SCAN_ITEMS <= NG) {
        uint4 *dst = reinterpret_cast<uint4 *>(kp.gstart + g0);
#pragma unroll
        for (int r = 0; r < SCAN_ITEMS / 4; ++r) dst[r] = make_uint4(out[4 * r], out[4 * r + 1], out[4 * r + 2], out[4 * r + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i)
            if (g0 + i < NG) kp.gstart[g0 + i] = out[i];
    }
    const int64_t base = (int64_t)tile * SCAN_TILE;
    if (base + SCAN_TILE >= NG && base < NG && threadIdx.x == 0) kp.gstart[NG] = (uint32_t)s_prefix + tile_total;
}

// ---------------------------------------------------------------------------
// Adds a0 to t[g0] and a1 to t[g1]. Adjacent nodes (g1 = g0 + 1) inside one
// aligned 8- or 16-byte block go in one vector reduction (zeros added to the
// other two floats of a 16-byte block), which halves the atomic operations
// of the deposit at the L2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_nodes(float *t, int64_t g0, int64_t g1, float a0, float a1)
{
    float *p = t + g0;
    const unsigned off = (unsigned)((reinterpret_cast<uintptr_t>(p) >> 2) & 3u);  // float slot in its 16 bytes
    if (g1 == g0 + 1 && (off & 1u) == 0u) {
        asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a0), "f"(a1) : "memory");
    } else if (g1 == g0 + 1 && off == 1u) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p - 1), "f"(0.f), "f"(a0), "f"(a1),
                     "f"(0.f)
                     : "memory");
    } else {
        atomicAdd(p, a0);
        atomicAdd(t + g1, a1);
    }
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
    else k0 = layer_of(kp, u);
    const bool walls = kp.pde_bc != 2;
    // the two nodes of each (y, z) row of the cell, x = i0 and i1
#pragma unroll
    for (int m = 0; m < (1 << (DIM - 1)); ++m) {
        const int by = m & 1, bz = (m >> 1) & 1;
        const int y = by ? j1 : j0, z = bz ? k1 : k0;
        float wr = by ? fy : 1.f - fy;
        if (DIM == 3) wr *= bz ? fz : 1.f - fz;
        if (walls) {
            if (y == 0 || y == kp.g[1] - 1) wr *= 2.f;
            if (DIM == 3 && ((z == 0 && !(kp.open_z & 1)) || (z == kp.g[2] - 1 && !(kp.open_z & 2)))) wr *= 2.f;
        }
        float w0 = (1.f - fx) * wr, w1 = fx * wr;
        if (walls) {
            if (i0 == 0) w0 *= 2.f;
            if (i1 == kp.g[0] - 1) w1 *= 2.f;
        }
        const int64_t g0 = gidx(kp, i0, y, z), g1 = gidx(kp, i1, y, z);
        if (fused) {
            float a0 = ks * w0, a1 = ks * w1;
            if (kc != 0.f) {
                a0 -= kp.dt * kc * w0 * __ldg(&cin[g0]);
                a1 -= kp.dt * kc * w1 * __ldg(&cin[g1]);
            }
            red_nodes(tS, g0, g1, a0, a1);
        } else {
            if (ks != 0.f) red_nodes(tS, g0, g1, ks * w0, ks * w1);
            if (kc != 0.f) red_nodes(tR, g0, g1, kc * w0, kc * w1);
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
    if (kp.Fh) {
        // half-window force sums, read by the particle kernel: cleared here for
        // the next step (a kernel that stores them without loading them first;
        // clearing right after the load in the particle kernel stalled it)
        longlong2 *pf = reinterpret_cast<longlong2 *>(kp.Fh + (size_t)j * FhStride<DIM>::value);
        pf[0] = make_longlong2(0ll, 0ll);
        if (DIM == 3) pf[1] = make_longlong2(0ll, 0ll);
    }
    const float4 u = kp.U[j];
    const uint32_t dst = bin_start(kp.cnt_nxt, kp.gstart, key_of(kp, u)) + kp.slot[j];
    if ((int64_t)dst >= kp.n) {
        set_err(kp, ERR_OVERFLOW);
        return;
    }
    kp.S[dst] = u;
    if (kp.dS) kp.dS[dst] = kp.dU[j];
    if (advance && kp.has_grid && kp.chem_mode == 0 && !kp.kde &&
        !(kp.sub && (__float_as_uint(u.w) & ID_MASK) == ID_MASK)) {  // a ghost's owner deposits it
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
// k_pde_stream: the same substep as k_pde, streamed. Each thread owns four
// consecutive x nodes (one float4) of a row and marches along the last axis
// (z in 3D, y in 2D), keeping the previous / current / next planes in
// registers; x neighbours come from the adjacent lanes (shuffles) and, in 3D,
// the y neighbours from the rows beside it (cache hits). One DRAM read and one
// write per node. Needs gx % 4 == 0.
// ---------------------------------------------------------------------------
template <int BC>
__device__ __forceinline__ int ghost(int k, int N)  // ghost rule along one axis
{
    if (BC == 2) return k < 0 ? k + N : (k >= N ? k - N : k);
    return k < 0 ? -k : (k > N - 1 ? 2 * (N - 1) - k : k);
}

__device__ __forceinline__ float4 f4_axpy(float a, float4 x, float4 y)
{
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

template <int DIM, int BC>
__global__ void __launch_bounds__(256) k_pde_stream(KP kp, const float *__restrict__ cin, float *__restrict__ cout,
                                                    int use_src, int last, int chunk)
{
    const int gx = kp.g[0], gy = kp.g[1], gz = DIM == 3 ? kp.g[2] : 1;
    const int nq = gx >> 2;
    const int lane = threadIdx.x;
    const int q = blockIdx.x * 32 + lane;
    const int qq = q < nq ? q : nq - 1;
    int y, s0, ns;
    if (DIM == 3) {
        y = blockIdx.y * blockDim.y + threadIdx.y;
        ns = gz;
        s0 = blockIdx.z * chunk;
    } else {
        y = 0;
        ns = gy;
        s0 = (blockIdx.z * blockDim.y + threadIdx.y) * chunk;
    }
    const bool active = q < nq && (DIM == 2 || y < gy);
    const int yy = DIM == 3 ? min(y, gy - 1) : 0;
    const int s1 = min(s0 + chunk, ns);
    if (s0 >= ns) return;  // whole warp (s0 depends on warp / block only)
    const int64_t sstride = DIM == 3 ? (int64_t)gx * gy : (int64_t)gx;
    // 2D: blockIdx.y is the layer (replicate) of the grid
    const int64_t rowbase = (DIM == 3 ? (int64_t)yy * gx : (int64_t)blockIdx.y * gx * gy) + 4 * (int64_t)qq;
    int64_t oym = 0, oyp = 0;
    if (DIM == 3) {
        oym = (int64_t)(ghost<BC>(yy - 1, gy) - yy) * gx;
        oyp = (int64_t)(ghost<BC>(yy + 1, gy) - yy) * gx;
    }
    const float ihx = kp.inv_h2[0], ihy = kp.inv_h2[1], ihz = kp.inv_h2[2];
    const float ihs = DIM == 3 ? ihz : ihy;  // stream axis
    const float Dc = kp.Dc, gam = kp.gamma, dts = kp.dts;
    const float inv_s = 1.f / (float)kp.substeps;
    const bool xlo = 4 * qq == 0, xhi = 4 * qq + 4 == gx;
    const bool ywall = DIM == 3 && (yy == 0 || yy == gy - 1);
    auto ld = [&](int64_t i) { return __ldg(reinterpret_cast<const float4 *>(cin + i)); };
    float4 vm = ld(rowbase + (int64_t)ghost<BC>(s0 - 1, ns) * sstride);
    float4 v0 = ld(rowbase + (int64_t)s0 * sstride);
    float4 vp = ld(rowbase + (int64_t)ghost<BC>(s0 + 1, ns) * sstride);
    for (int s = s0; s < s1; ++s) {
        const int64_t b = rowbase + (int64_t)s * sstride;
        const float4 vq = (s + 1 < s1) ? ld(rowbase + (int64_t)ghost<BC>(s + 2, ns) * sstride) : vp;
        float left = __shfl_up_sync(0xffffffffu, v0.w, 1);
        float right = __shfl_down_sync(0xffffffffu, v0.x, 1);
        if (xlo) left = BC == 2 ? __ldg(cin + b + gx - 1) : v0.y;
        else if (lane == 0) left = __ldg(cin + b - 1);
        if (xhi) right = BC == 2 ? __ldg(cin + b - (gx - 4)) : v0.z;
        else if (lane == 31) right = __ldg(cin + b + 4);
        float4 lap;
        lap.x = (left + v0.y - 2.f * v0.x) * ihx;
        lap.y = (v0.x + v0.z - 2.f * v0.y) * ihx;
        lap.z = (v0.y + v0.w - 2.f * v0.z) * ihx;
        lap.w = (v0.z + right - 2.f * v0.w) * ihx;
        lap.x = fmaf(vm.x + vp.x - 2.f * v0.x, ihs, lap.x);
        lap.y = fmaf(vm.y + vp.y - 2.f * v0.y, ihs, lap.y);
        lap.z = fmaf(vm.z + vp.z - 2.f * v0.z, ihs, lap.z);
        lap.w = fmaf(vm.w + vp.w - 2.f * v0.w, ihs, lap.w);
        if (DIM == 3) {
            const float4 a = ld(b + oym), c = ld(b + oyp);
            lap.x = fmaf(a.x + c.x - 2.f * v0.x, ihy, lap.x);
            lap.y = fmaf(a.y + c.y - 2.f * v0.y, ihy, lap.y);
            lap.z = fmaf(a.z + c.z - 2.f * v0.z, ihy, lap.z);
            lap.w = fmaf(a.w + c.w - 2.f * v0.w, ihy, lap.w);
        }
        // rhs = D_c lap - gamma c - R c
        float4 rhs = make_float4(Dc * lap.x - gam * v0.x, Dc * lap.y - gam * v0.y, Dc * lap.z - gam * v0.z,
                                 Dc * lap.w - gam * v0.w);
        float4 add = make_float4(0.f, 0.f, 0.f, 0.f);
        if (use_src) {
            float4 *S4 = reinterpret_cast<float4 *>(kp.srcg + b);
            float4 *R4 = reinterpret_cast<float4 *>(kp.Rg + b);
            const float4 Sv = *S4, Rv = *R4;
            rhs.x -= Rv.x * v0.x;
            rhs.y -= Rv.y * v0.y;
            rhs.z -= Rv.z * v0.z;
            rhs.w -= Rv.w * v0.w;
            add = make_float4(Sv.x * inv_s, Sv.y * inv_s, Sv.z * inv_s, Sv.w * inv_s);
            if (last && active) {
                *S4 = make_float4(0.f, 0.f, 0.f, 0.f);
                *R4 = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float4 out = f4_axpy(dts, rhs, make_float4(v0.x + add.x, v0.y + add.y, v0.z + add.z, v0.w + add.w));
        if (BC == 1) {  // Dirichlet: wall nodes keep their value
            const bool swall = s == 0 || s == ns - 1;
            if (swall || ywall) out = v0;
            if (xlo) out.x = v0.x;
            if (xhi) out.w = v0.w;
        }
        if (active) *reinterpret_cast<float4 *>(cout + b) = out;
        vm = v0;
        v0 = vp;
        vp = vq;
    }
}

// ---------------------------------------------------------------------------
// k_pde_multi: up to PDE_MULTI_MAX substeps of Eq. (1d) on a 2D grid in one
// launch (temporal blocking). A block owns a PM_T x PM_T tile of nodes and
// loads it with a halo of nsub nodes into shared memory: the mirror-ghost
// (Neumann) problem is exactly the problem on the mirror-extended grid with
// mirror-extended data and sources, so the halo is filled by reflecting the
// node index (periodic: wrapping; Dirichlet: wall nodes are held and the
// halo beyond them is never used). Each substep updates every node but the
// outer ring of the tile; the stale ring reaches one node further in per
// substep, never the tile itself.
// ---------------------------------------------------------------------------
constexpr int PM_T = 32;
constexpr int PM_TPB = 1024;  // one thread per output node
constexpr int PM_ROWS = PM_TPB / 32;

__device__ __forceinline__ int pm_map(int k, int N, int bc)
{
    if (bc == 2) {
        k %= N;
        return k < 0 ? k + N : k;
    }
    if (bc == 1) return k < 0 ? 0 : (k > N - 1 ? N - 1 : k);
    const int P = 2 * (N - 1);  // mirror: the index reflects with period 2 (N - 1)
    k %= P;
    if (k < 0) k += P;
    return k > N - 1 ? P - k : k;
}

template <int BC>
__global__ void __launch_bounds__(PM_TPB) k_pde_multi(KP kp, const float *__restrict__ cin, float *__restrict__ cout,
                                                      int nsub, int use_src, float *__restrict__ avg, int avg_first,
                                                      float avg_scale, int tau_mode)
{
    extern __shared__ float pm[];
    // threads as 32 columns x PM_ROWS rows; the tile is W x W, W = PM_T + 2 nsub <= 56
    const int H = nsub, W = PM_T + 2 * nsub, WW = W * W;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    float *A = pm, *B = pm + WW;
    float *Sv = pm + 2 * WW, *Rv = pm + 3 * WW;
    const int gx = kp.g[0], gy = kp.g[1];
    const int x0 = blockIdx.x * PM_T - H, y0 = blockIdx.y * PM_T - H;
    const int64_t lbase = (int64_t)blockIdx.z * gx * gy;  // layer of an ensemble
    for (int ty = ly; ty < W; ty += PM_ROWS) {
        const int my = pm_map(y0 + ty, gy, BC);
        const bool ywall = my == 0 || my == gy - 1;
        for (int tx = lx; tx < W; tx += 32) {
            const int mx = pm_map(x0 + tx, gx, BC);
            const int64_t g = lbase + (int64_t)my * gx + mx;
            float v = cin[g];
            if (tau_mode && BC != 2) {  // c / tau: tau = 1/2 per wall axis
                if (mx == 0 || mx == gx - 1) v *= 2.f;
                if (ywall) v *= 2.f;
            }
            const int i = ty * W + tx;
            A[i] = v;
            if (use_src) {
                Sv[i] = kp.srcg[g];
                Rv[i] = kp.Rg[g];
            }
        }
    }
    constexpr int OWN = PM_T * PM_T / PM_TPB;  // output nodes per thread: column lx, rows ly + PM_ROWS q
    float acc[OWN];
#pragma unroll
    for (int q = 0; q < OWN; ++q) acc[q] = 0.f;
    const float ihx = kp.inv_h2[0], ihy = kp.inv_h2[1], Dc = kp.Dc, gam = kp.gamma, dts = kp.dts;
    const float inv_s = 1.f / (float)kp.substeps;
    for (int m = 0; m < nsub; ++m) {
        __syncthreads();
        if (avg) {
#pragma unroll
            for (int q = 0; q < OWN; ++q) acc[q] += A[(ly + PM_ROWS * q + H) * W + lx + H];
        }
        // nodes that can still reach the output tile: [m + 1, W - m - 1)
        const int lo = m + 1, hi = W - m - 1;
        for (int ty = lo + ly; ty < hi; ty += PM_ROWS) {
            for (int tx = lo + lx; tx < hi; tx += 32) {
                const int i = ty * W + tx;
                const float c = A[i];
                const float lap = (A[i - 1] + A[i + 1] - 2.f * c) * ihx + (A[i - W] + A[i + W] - 2.f * c) * ihy;
                float rhs = Dc * lap - gam * c;
                float add = 0.f;
                if (use_src) {
                    rhs -= Rv[i] * c;
                    add = Sv[i] * inv_s;
                }
                float out = fmaf(dts, rhs, c + add);
                if (BC == 1) {  // Dirichlet: wall nodes keep their value
                    const int X = x0 + tx, Y = y0 + ty;
                    if (X <= 0 || Y <= 0 || X >= gx - 1 || Y >= gy - 1) out = c;
                }
                B[i] = out;
            }
        }
        float *tmp = A;
        A = B;
        B = tmp;
    }
    __syncthreads();
    const int X = blockIdx.x * PM_T + lx;
#pragma unroll
    for (int q = 0; q < OWN; ++q) {
        const int oy = ly + PM_ROWS * q;
        const int Y = blockIdx.y * PM_T + oy;
        if (X >= gx || Y >= gy) continue;
        float v = A[(oy + H) * W + lx + H];
        if (tau_mode && BC != 2) {
            float t = 1.f;
            if (X == 0 || X == gx - 1) t *= 0.5f;
            if (Y == 0 || Y == gy - 1) t *= 0.5f;
            v *= t;
        }
        const int64_t g = lbase + (int64_t)Y * gx + X;
        cout[g] = v;
        if (avg) avg[g] = avg_first ? acc[q] * avg_scale : fmaf(acc[q], avg_scale, avg[g]);
    }
}

// ---------------------------------------------------------------------------
// Hard-sphere overlap correction (Sect. 3.2) of the moved, sorted cells:
// every pair closer than its contact distance is pushed apart along the line
// of centres by twice the penetration, cell i taking D_i / (D_i + D_j) of
// it; all corrections come from the moved positions, then the boundary rule
// again. The corrected cells go to U with their bins counted for the next
// sort (as after the particle kernel).
// ---------------------------------------------------------------------------
constexpr int HS_TPC = 4;  // threads per cell of the correction (consecutive lanes)

template <int DIM, bool PERIODIC>
__global__ void __launch_bounds__(TPB) k_hard_sphere(KP kp)
{
    const int64_t t = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const int64_t j = t / HS_TPC;
    const int sub = (int)(t % HS_TPC);
    const bool valid = j < kp.n;
    const float4 me = valid ? kp.S[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t w = __float_as_uint(me.w);
    const int sp = (int)(w >> SP_SHIFT);
    float acc[3] = {0.f, 0.f, 0.f};
    if (valid) {
        int c[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        const float pc[3] = {me.x, me.y, me.z};
        for (int a = 0; a < DIM; ++a) {
            c[a] = bin_axis(pc[a], kp.lo[a], kp.inv_b[a], kp.nb[a]);
            lo[a] = c[a] - 1;
            hi[a] = c[a] + 1;
            if (!PERIODIC) {
                lo[a] = max(lo[a], 0);
                hi[a] = min(hi[a], kp.nb[a] - 1);
            }
        }
        if (DIM == 2) lo[2] = hi[2] = layer_of(kp, me);
        const uint32_t n = (uint32_t)kp.n;
        for (int z = lo[2]; z <= hi[2]; ++z) {
            const int zz = (PERIODIC && DIM == 3) ? (z < 0 ? z + kp.nb[2] : (z >= kp.nb[2] ? z - kp.nb[2] : z)) : z;
            for (int y = lo[1]; y <= hi[1]; ++y) {
                const int yy = PERIODIC ? (y < 0 ? y + kp.nb[1] : (y >= kp.nb[1] ? y - kp.nb[1] : y)) : y;
                const uint32_t rowk = (uint32_t)kp.px * ((uint32_t)yy + (uint32_t)kp.nb[1] * (uint32_t)zz);
                // the row's bins as contiguous ranges (a wrapped periodic row is two)
                int xa[2] = {lo[0], 0}, xb[2] = {hi[0], -1};
                if (PERIODIC && lo[0] < 0) {
                    xa[0] = 0;
                    xa[1] = xb[1] = kp.nb[0] + lo[0];
                } else if (PERIODIC && hi[0] >= kp.nb[0]) {
                    xb[0] = kp.nb[0] - 1;
                    xa[1] = 0;
                    xb[1] = hi[0] - kp.nb[0];
                }
                for (int piece = 0; piece < 2; ++piece) {
                    if (xa[piece] > xb[piece]) continue;
                    const uint32_t q0 = min(bin_start(kp.cnt_cur, kp.gstart, rowk + (uint32_t)xa[piece]), n);
                    const uint32_t q1 = min(bin_start(kp.cnt_cur, kp.gstart, rowk + (uint32_t)xb[piece] + 1u), n);
                    for (uint32_t q = q0 + (uint32_t)sub; q < q1; q += HS_TPC) {
                        if (q == (uint32_t)j) continue;
                        const float4 o = __ldg(&kp.S[q]);
                        float dx, dy, dz, r2;
                        pair_delta<DIM, PERIODIC>(kp, me, o, dx, dy, dz, r2);
                        const int st = sp * MAXS + (int)(__float_as_uint(o.w) >> SP_SHIFT);
                        const float contact = kp.hs_contact[st];
                        if (!(r2 > 0.f) || !(r2 < contact * contact)) continue;
                        const float r = sqrtf(r2);
                        const float move = 2.f * (contact - r) * kp.hs_share[st] / r;
                        acc[0] = fmaf(move, dx, acc[0]);
                        acc[1] = fmaf(move, dy, acc[1]);
                        if (DIM == 3) acc[2] = fmaf(move, dz, acc[2]);
                    }
                }
            }
        }
    }
    // the HS_TPC threads of a cell are consecutive lanes of one warp
    for (int o = HS_TPC / 2; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if (!valid || sub != 0) return;
    const float x1 = me.x + acc[0], y1 = me.y + acc[1], z1 = DIM == 3 ? me.z + acc[2] : me.z;
    float xb, yb, zb;
    if (PERIODIC) {
        xb = wrap_axis(x1, kp.lo[0], kp.hi[0], kp.L[0]);
        yb = wrap_axis(y1, kp.lo[1], kp.hi[1], kp.L[1]);
        zb = DIM == 3 ? wrap_axis(z1, kp.lo[2], kp.hi[2], kp.L[2]) : me.z;
    } else {
        xb = reflect_axis(x1, kp.lo[0], kp.hi[0]);
        yb = reflect_axis(y1, kp.lo[1], kp.hi[1]);
        zb = DIM == 3 ? reflect_axis(z1, kp.lo[2], kp.hi[2]) : me.z;
    }
    if (kp.dS) {
        float4 d = kp.dS[j];
        if (PERIODIC) {
            d.x += acc[0];
            d.y += acc[1];
            d.z += DIM == 3 ? acc[2] : 0.f;
        } else {
            d.x += xb - me.x;
            d.y += yb - me.y;
            d.z += DIM == 3 ? zb - me.z : 0.f;
        }
        kp.dU[j] = d;
    }
    const float4 nu = make_float4(xb, yb, zb, me.w);
    kp.U[j] = nu;
    kp.slot[j] = count_bin(kp.cnt_nxt, key_of(kp, nu), kp.err);
}

// ---------------------------------------------------------------------------
// Gaussian kernel density estimate at the grid nodes (Sect. 2.3; the density
// listing of Sect. 3): node l gathers, through the cell list of the sorted
// state, the cells within kde_range bandwidths, K_s(x) = (2 pi sigma_s^2)^
// (-d/2) exp(-|x|^2 / (2 sigma_s^2)), and writes the source dt sum k_s K_s
// and the consumption sum kappa_s K_s. Only the bins that meet the sphere of
// the largest truncation radius are visited: rows farther away are skipped
// and each row is cut to one contiguous x-range. The sums are exact (32-bit
// fixed point, 2^-24 of the largest term, folded into 64 bits every 64
// terms), so the result does not depend on the order of the cells in a bin.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kde_gap(float p, float lo, float b, int k, int c)
{
    if (k == c) return 0.f;
    return k < c ? p - (lo + (float)(k + 1) * b) : (lo + (float)k * b) - p;
}

template <int DIM, bool PERIODIC>
__global__ void __launch_bounds__(TPB) k_kde(KP kp, float *__restrict__ S_out, float *__restrict__ R_out)
{
    const int64_t g = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (g >= kp.G) return;
    const int gx = kp.g[0], gy = kp.g[1];
    const int ix = (int)(g % gx);
    const int iy = (int)((g / gx) % gy);
    const int iz = (int)(g / ((int64_t)gx * gy));  // plane (3D) or layer (2D)
    // node position as a float pair hi + lo (the steep kernel magnifies the
    // rounding of a single float node coordinate): the difference to a cell
    // is (hi - x) + lo
    const int ik[3] = {ix, iy, iz};
    float node[3] = {0.f, 0.f, (float)iz}, nlo[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < DIM; ++a) {
        const double v = kp.lo_d[a] + (double)ik[a] * kp.hgrid_d[a];
        node[a] = (float)v;
        nlo[a] = (float)(v - (double)node[a]);
    }
    const float4 me = make_float4(node[0], node[1], node[2], 0.f);
    const int W = kp.kde_win;
    const float R = kp.kde_rmax, R2 = R * R;
    int c[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a) {
        c[a] = bin_axis(node[a], kp.lo[a], kp.inv_b[a], kp.nb[a]);
        lo[a] = c[a] - W;
        hi[a] = c[a] + W;
        if (!PERIODIC) {
            lo[a] = max(lo[a], 0);
            hi[a] = min(hi[a], kp.nb[a] - 1);
        }
    }
    if (DIM == 2) lo[2] = hi[2] = c[2] = min(max(iz, 0), kp.layers - 1);
    long long accS = 0, accR = 0;
    int accS32 = 0, accR32 = 0, nterm = 0;
    const uint32_t n = (uint32_t)kp.n;
    for (int z = lo[2]; z <= hi[2]; ++z) {
        const float gz = DIM == 3 ? kde_gap(node[2], kp.lo[2], kp.bside[2], z, c[2]) : 0.f;
        const int zz = (PERIODIC && DIM == 3) ? (z < 0 ? z + kp.nb[2] : (z >= kp.nb[2] ? z - kp.nb[2] : z)) : z;
        for (int y = lo[1]; y <= hi[1]; ++y) {
            const float gyv = kde_gap(node[1], kp.lo[1], kp.bside[1], y, c[1]);
            const float g2 = gyv * gyv + gz * gz;
            if (!(g2 < R2)) continue;  // the row misses the sphere
            const int yy = PERIODIC ? (y < 0 ? y + kp.nb[1] : (y >= kp.nb[1] ? y - kp.nb[1] : y)) : y;
            const uint32_t rowk = (uint32_t)kp.px * ((uint32_t)yy + (uint32_t)kp.nb[1] * (uint32_t)zz);
            // x-bins that meet the sphere's section with this row
            const float ext = sqrtf(R2 - g2) + 1e-4f * kp.bside[0];  // margin over the rounding of bin edges
            int x0 = (int)floorf((node[0] - ext - kp.lo[0]) * kp.inv_b[0]);
            int x1 = (int)floorf((node[0] + ext - kp.lo[0]) * kp.inv_b[0]);
            x0 = max(x0, lo[0]);
            x1 = min(x1, hi[0]);
            int xa[2] = {x0, 0}, xb[2] = {x1, -1};
            if (PERIODIC && x0 < 0) {
                xa[0] = 0;
                xa[1] = x0 + kp.nb[0];
                xb[1] = kp.nb[0] - 1;
            } else if (PERIODIC && x1 >= kp.nb[0]) {
                xb[0] = kp.nb[0] - 1;
                xa[1] = 0;
                xb[1] = x1 - kp.nb[0];
            }
            for (int piece = 0; piece < 2; ++piece) {
                if (xa[piece] > xb[piece]) continue;
                const uint32_t q0 = min(bin_start(kp.cnt_cur, kp.gstart, rowk + (uint32_t)xa[piece]), n);
                const uint32_t q1 = min(bin_start(kp.cnt_cur, kp.gstart, rowk + (uint32_t)xb[piece] + 1u), n);
                for (uint32_t q = q0; q < q1; ++q) {
                    const float4 o = __ldg(&kp.S[q]);
                    const int s = (int)(__float_as_uint(o.w) >> SP_SHIFT);
                    float dx, dy, dz, r2;
                    pair_delta<DIM, PERIODIC>(kp, me, o, dx, dy, dz, r2);
                    dx += nlo[0];
                    dy += nlo[1];
                    dz = DIM == 3 ? dz + nlo[2] : 0.f;
                    r2 = DIM == 3 ? fmaf(dx, dx, fmaf(dy, dy, dz * dz)) : fmaf(dx, dx, dy * dy);
                    if (!(r2 < kp.kde_r2[s])) continue;
                    const float e = __expf(-r2 * kp.kde_c[s]);
                    accS32 += __float2int_rn(kp.kde_src[s] * e * kp.kde_qs_inv);
                    accR32 += __float2int_rn(kp.kde_cons[s] * e * kp.kde_qr_inv);
                    if (++nterm == 64) {  // terms are below 2^24: 64 of them fit an int32
                        accS += accS32;
                        accR += accR32;
                        accS32 = accR32 = nterm = 0;
                    }
                }
            }
        }
    }
    accS += accS32;
    accR += accR32;
    S_out[g] = (float)((double)accS * (double)kp.kde_qs);
    if (R_out) R_out[g] = (float)((double)accR * (double)kp.kde_qr);
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
    const int64_t id = gid_of(kp, u);
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

// Initial state of the paper's experiments (Sect. 3): cell i < n_alpha is
// species 0 (alpha), drawn from a normal distribution centred in the box with
// standard deviation sigma_frac x the box width per axis and put inside by
// the box's boundary rule (reflection or wrap); the other cells are species
// 1 (beta), uniform in the box. Philox words of counter (i, 0, TAG_INIT, 0)
// under the key (seed lo, seed hi); Box-Muller as for the move's noise.
__global__ void k_init_positions(int dim, int periodic, float3 lo3, float3 hi3, int64_t n, int64_t n_alpha,
                                 float sigma_frac, uint32_t k0, uint32_t k1, float *__restrict__ pos,
                                 uint8_t *__restrict__ sp)
{
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0u, TAG_INIT, 0u), k0, k1);
    const float lo[3] = {lo3.x, lo3.y, lo3.z}, hi[3] = {hi3.x, hi3.y, hi3.z};
    const bool alpha = i < n_alpha;
    float g[3] = {0.f, 0.f, 0.f};
    if (alpha) {
        const float2 a = box_muller(w.x, w.y);
        g[0] = a.x;
        g[1] = a.y;
        g[2] = box_muller(w.z, w.w).x;
    }
    const uint32_t ws[3] = {w.x, w.y, w.z};
    for (int a = 0; a < dim; ++a) {
        const float L = hi[a] - lo[a];
        float x;
        if (alpha) {
            x = fmaf(sigma_frac * L, g[a], 0.5f * (lo[a] + hi[a]));
            x = periodic ? wrap_axis(x, lo[a], hi[a], L) : reflect_axis(x, lo[a], hi[a]);
        } else {
            x = fmaf(word_uniform(ws[a]), L, lo[a]);
            if (periodic && x >= hi[a]) x = lo[a];
        }
        pos[i * dim + a] = x;
    }
    sp[i] = alpha ? 0 : 1;
}

__global__ void k_stage_bins(KP kp, int32_t *__restrict__ cells)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 u = kp.S[j];
    const int64_t id = gid_of(kp, u);
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
    if (j < kp.n) ids[j] = (uint32_t)gid_of(kp, kp.S[j]);
}

// Offset of every bin (bin_slots + 1 entries) of the sorted state.
__global__ void k_stage_starts(KP kp, uint32_t *__restrict__ out)
{
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k <= kp.bin_slots) out[k] = bin_start(kp.cnt_cur, kp.gstart, (uint32_t)k);
}

template <int DIM, bool PERIODIC, bool WARP>
__global__ void __launch_bounds__(TPB, CHEMO_PAIR_BLOCKS) k_stage_forces(KP kp, float *__restrict__ F_out, int32_t *__restrict__ count,
                                                      unsigned long long *__restrict__ idsum)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemTables &t = *reinterpret_cast<SmemTables *>(smem);
    load_tables(kp, t);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const bool valid = j < kp.n;
    const float4 me = valid ? kp.S[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t w = __float_as_uint(me.w);
    const int64_t id = valid ? gid_of(kp, me) : 0;
    int cnt = 0;
    unsigned long long ids = 0ull;
    float3 F = make_float3(0.f, 0.f, 0.f);
    if (kp.pairs) {  // warp-synchronous: every lane takes part
        unsigned char *wbuf = smem + sizeof(SmemTables) + (threadIdx.x >> 5) * warp_region<DIM, PERIODIC, WARP>();
        if (WARP)
            F = pair_force_warp<DIM, PERIODIC, true>(kp, t, wbuf, (uint32_t)j, me, (int)(w >> SP_SHIFT), valid, cnt,
                                                     ids);
        else
            F = pair_force<DIM, PERIODIC, true>(kp, t, (uint32_t)j, me, (int)(w >> SP_SHIFT), valid, cnt, ids, wbuf);
    }
    if (!valid) return;
    if (id >= kp.n) {
        set_err(kp, ERR_OVERFLOW);
        return;
    }
    F_out[id * DIM + 0] = F.x;
    F_out[id * DIM + 1] = F.y;
    if (DIM == 3) F_out[id * DIM + 2] = F.z;
    if (count) count[id] = cnt;
    if (idsum) idsum[id] = ids;
}

// The half-window kernel's force sums by id (search mode 4), cleared after
// (a test entry point: the step clears them in the scatter).
template <int DIM>
__global__ void k_stage_take_half(KP kp, float *__restrict__ F_out)
{
    constexpr int FS = FhStride<DIM>::value;
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const int64_t id = gid_of(kp, kp.S[j]);
    long long *pf = kp.Fh + (size_t)j * FS;
    for (int a = 0; a < DIM; ++a) {
        const long long v = pf[a];
        pf[a] = 0ll;
        if (id < kp.n) F_out[id * DIM + a] = __ll2float_rn(v) * kp.fq;
    }
}

template <int DIM>
__global__ void k_stage_drift(KP kp, int cur, float *__restrict__ out)
{
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 me = kp.S[j];
    const uint32_t w = __float_as_uint(me.w);
    const int64_t id = gid_of(kp, me);
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

// Pair kernels may need more than the default 48 KB of dynamic shared memory.
// The pair kernels run CHEMO_PAIR_BLOCKS blocks per SM (register bound). Ask for just the
// shared memory those blocks need and leave the rest of the SM's 256 KB to
// L1, which caches the candidate positions.
template <typename K>
static void allow_smem(K kernel, size_t bytes, int blocks = CHEMO_PAIR_BLOCKS)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    const double need = (double)blocks * (double)(bytes + 1024) / (228.0 * 1024.0);
    const int pct = (int)std::ceil(100.0 * need);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct > 100 ? 100 : pct);
}

template <bool W>
static void pair_kernel_attributes_of()
{
    allow_smem(k_step<2, false, W>, pair_smem<2, false, W>());
    allow_smem(k_step<2, true, W>, pair_smem<2, true, W>());
    allow_smem(k_step<3, false, W>, pair_smem<3, false, W>());
    allow_smem(k_step<3, true, W>, pair_smem<3, true, W>());
    allow_smem(k_stage_forces<2, false, W>, pair_smem<2, false, W>());
    allow_smem(k_stage_forces<2, true, W>, pair_smem<2, true, W>());
    allow_smem(k_stage_forces<3, false, W>, pair_smem<3, false, W>());
    allow_smem(k_stage_forces<3, true, W>, pair_smem<3, true, W>());
}

template <int BT>
static void half_block_attributes()
{
    constexpr int nb = CHEMO_PAIR_BLOCKS * TPB / BT;
    allow_smem(k_pairs_half<2, false, BT>, pair_smem<2, false, false, BT>(), nb);
    allow_smem(k_pairs_half<2, true, BT>, pair_smem<2, true, false, BT>(), nb);
    allow_smem(k_pairs_half<3, false, BT>, pair_smem<3, false, false, BT>(), nb);
    allow_smem(k_pairs_half<3, true, BT>, pair_smem<3, true, false, BT>(), nb);
}

static void pair_kernel_attributes()
{
    static bool done = false;
    if (done) return;
    pair_kernel_attributes_of<false>();
    pair_kernel_attributes_of<true>();
    allow_smem(k_pairs_half<2, false>, pair_smem<2, false, false>());
    allow_smem(k_pairs_half<2, true>, pair_smem<2, true, false>());
    allow_smem(k_pairs_half<3, false>, pair_smem<3, false, false>());
    allow_smem(k_pairs_half<3, true>, pair_smem<3, true, false>());
    half_block_attributes<128>();
    half_block_attributes<512>();
    done = true;
}

// The 3^d window uses the warp search, the 2^d window the per-lane search.
// The half-window pair kernel and the move kernel after it, BT threads per block.
template <int DIM, bool PERIODIC, int BT>
static void half_step_launch(const KP &kp, int cur, cudaStream_t st)
{
    const unsigned nb = (unsigned)((kp.n + BT - 1) / BT);
    k_pairs_half<DIM, PERIODIC, BT><<<nb, BT, pair_smem<DIM, PERIODIC, false, BT>(), st>>>(kp);
    k_step<DIM, PERIODIC, false, true, BT><<<nb, BT, sizeof(SmemTables), st>>>(kp, cur);
}

template <int DIM, bool PERIODIC>
static void half_pairs_launch(const KP &kp, cudaStream_t st)
{
    if (kp.bt == 128)
        k_pairs_half<DIM, PERIODIC, 128><<<(unsigned)((kp.n + 127) / 128), 128, pair_smem<DIM, PERIODIC, false, 128>(), st>>>(kp);
    else if (kp.bt == 512)
        k_pairs_half<DIM, PERIODIC, 512><<<(unsigned)((kp.n + 511) / 512), 512, pair_smem<DIM, PERIODIC, false, 512>(), st>>>(kp);
    else
        k_pairs_half<DIM, PERIODIC><<<(unsigned)((kp.n + TPB - 1) / TPB), TPB, pair_smem<DIM, PERIODIC, false>(), st>>>(kp);
}

template <int DIM, bool PERIODIC, bool W>
static void step_launch(const KP &kp, int cur, cudaStream_t st)
{
    const unsigned nb = (unsigned)((kp.n + TPB - 1) / TPB);
    if (kp.pairs && kp.Fh) {
        if (kp.bt == 128) half_step_launch<DIM, PERIODIC, 128>(kp, cur, st);
        else if (kp.bt == 512) half_step_launch<DIM, PERIODIC, 512>(kp, cur, st);
        else half_step_launch<DIM, PERIODIC, TPB>(kp, cur, st);
    } else {
        k_step<DIM, PERIODIC, W><<<nb, TPB, pair_smem<DIM, PERIODIC, W>(), st>>>(kp, cur);
    }
}

cudaError_t launch_step_particles(const KP &kp, int cur, cudaStream_t st, int *launches)
{
    if (kp.n == 0) {  // no particle kernel: the source grids of the last step are cleared here
        if (kp.zero_src && kp.has_grid) {
            cudaError_t e = cudaMemsetAsync(kp.srcg, 0, (size_t)kp.G * sizeof(float), st);
            if (e == cudaSuccess) e = cudaMemsetAsync(kp.Rg, 0, (size_t)kp.G * sizeof(float), st);
            return e;
        }
        return cudaSuccess;
    }
    pair_kernel_attributes();
    if (launches && kp.pairs && kp.Fh) ++*launches;
    const bool w = kp.search == 1;
    if (kp.dim == 2) {
        if (kp.periodic) w ? step_launch<2, true, true>(kp, cur, st) : step_launch<2, true, false>(kp, cur, st);
        else w ? step_launch<2, false, true>(kp, cur, st) : step_launch<2, false, false>(kp, cur, st);
    } else {
        if (kp.periodic) w ? step_launch<3, true, true>(kp, cur, st) : step_launch<3, true, false>(kp, cur, st);
        else w ? step_launch<3, false, true>(kp, cur, st) : step_launch<3, false, false>(kp, cur, st);
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

unsigned scan_tiles(const KP &kp) { return (unsigned)((kp.ngroups + SCAN_TILE - 1) / SCAN_TILE); }

cudaError_t launch_scan(const KP &kp, cudaStream_t st, int *launches)
{
    const unsigned tiles = scan_tiles(kp);
    k_scan<<<tiles, TPB, 0, st>>>(kp);
    if (launches) ++*launches;
    return cudaGetLastError();
}

__global__ void k_set_tile_ctr(uint32_t *ctr, uint32_t v) { *ctr = v; }

__global__ void k_end_scan(uint32_t *ctr, uint32_t *seq)
{
    *ctr = 0u;
    *seq += 1u;
}

cudaError_t launch_scan_from_tile(const KP &kp, uint32_t first_tile, cudaStream_t st)
{
    k_set_tile_ctr<<<1, 1, 0, st>>>(kp.tile_ctr, first_tile);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_scan(kp, st, nullptr);
    if (e != cudaSuccess) return e;
    k_end_scan<<<1, 1, 0, st>>>(kp.tile_ctr, kp.scan_seq);
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

template <int DIM>
static void pde_stream_launch(const KP &kp, const float *cin, float *cout, int use_src, int last, cudaStream_t st)
{
    const int nq = kp.g[0] / 4;
    const int bx = (nq + 31) / 32;
    const dim3 block(32, 8);
    if (DIM == 3) {
        // aim at about four blocks per SM; chunks of at least 8 planes
        const int by = (kp.g[1] + 7) / 8;
        int chunk = 8;
        while (chunk < kp.g[2] && (int64_t)bx * by * ((kp.g[2] + 2 * chunk - 1) / (2 * chunk)) >= 608) chunk *= 2;
        const dim3 grid(bx, by, (kp.g[2] + chunk - 1) / chunk);
        if (kp.pde_bc == 0) k_pde_stream<3, 0><<<grid, block, 0, st>>>(kp, cin, cout, use_src, last, chunk);
        else if (kp.pde_bc == 1) k_pde_stream<3, 1><<<grid, block, 0, st>>>(kp, cin, cout, use_src, last, chunk);
        else k_pde_stream<3, 2><<<grid, block, 0, st>>>(kp, cin, cout, use_src, last, chunk);
    } else {
        int chunk = 4;
        while (chunk < kp.g[1] && (int64_t)bx * 8 * ((kp.g[1] + 2 * chunk - 1) / (2 * chunk)) >= 2432) chunk *= 2;
        const int warps = (kp.g[1] + chunk - 1) / chunk;
        const dim3 grid(bx, kp.g[2], (warps + 7) / 8);
        if (kp.pde_bc == 0) k_pde_stream<2, 0><<<grid, block, 0, st>>>(kp, cin, cout, use_src, last, chunk);
        else if (kp.pde_bc == 1) k_pde_stream<2, 1><<<grid, block, 0, st>>>(kp, cin, cout, use_src, last, chunk);
        else k_pde_stream<2, 2><<<grid, block, 0, st>>>(kp, cin, cout, use_src, last, chunk);
    }
}

static size_t pde_multi_smem(int nsub)
{
    const size_t W = (size_t)(PM_T + 2 * nsub);
    return 4 * W * W * sizeof(float);
}

cudaError_t launch_pde_multi(const KP &kp, const float *cin, float *cout, int nsub, int use_src, float *avg,
                             int avg_first, float avg_scale, int tau_mode, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        const int mx = (int)pde_multi_smem(PDE_MULTI_MAX);
        cudaFuncSetAttribute(k_pde_multi<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_pde_multi<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_pde_multi<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        attr = true;
    }
    if (nsub < 1 || nsub > PDE_MULTI_MAX) return cudaErrorInvalidValue;
    const dim3 grid((kp.g[0] + PM_T - 1) / PM_T, (kp.g[1] + PM_T - 1) / PM_T, kp.g[2]);
    const size_t sm = pde_multi_smem(nsub);
    if (kp.pde_bc == 0) k_pde_multi<0><<<grid, PM_TPB, sm, st>>>(kp, cin, cout, nsub, use_src, avg, avg_first, avg_scale, tau_mode);
    else if (kp.pde_bc == 1) k_pde_multi<1><<<grid, PM_TPB, sm, st>>>(kp, cin, cout, nsub, use_src, avg, avg_first, avg_scale, tau_mode);
    else k_pde_multi<2><<<grid, PM_TPB, sm, st>>>(kp, cin, cout, nsub, use_src, avg, avg_first, avg_scale, tau_mode);
    return cudaGetLastError();
}

cudaError_t launch_pde(const KP &kp, int cur, cudaStream_t st, int *launches)
{
    if (!kp.has_grid || kp.chem_mode != 0) return cudaSuccess;
    if (kp.pde_multi) {
        // the substeps split as evenly as possible over the launches
        int c = cur, left = kp.substeps;
        for (int l = 0; l < kp.pde_launches; ++l) {
            const int nsub = (left + (kp.pde_launches - l) - 1) / (kp.pde_launches - l);
            const cudaError_t e = launch_pde_multi(kp, kp.c[c], kp.c[c ^ 1], nsub, kp.fused_deposit ? 0 : 1, nullptr,
                                                   0, 0.f, 0, st);
            if (e != cudaSuccess) return e;
            left -= nsub;
            c ^= 1;
            if (launches) ++*launches;
        }
        return cudaSuccess;
    }
    const bool stream = kp.g[0] % 4 == 0 && kp.g[0] >= 8;
    const dim3 grid((kp.g[0] + 127) / 128, kp.g[1], kp.g[2]);  // g[2]: planes (3D) or layers (2D)
    const int s = kp.substeps;
    const int use_src = kp.fused_deposit ? 0 : 1;
    int c = cur;
    for (int m = 0; m < s; ++m) {
        const int last = m == s - 1 && !kp.zero_src;  // else the next particle kernel clears the sources
        if (stream) {
            if (kp.dim == 2) pde_stream_launch<2>(kp, kp.c[c], kp.c[c ^ 1], use_src, last, st);
            else pde_stream_launch<3>(kp, kp.c[c], kp.c[c ^ 1], use_src, last, st);
        } else if (kp.dim == 2) {
            k_pde<2><<<grid, 128, 0, st>>>(kp, kp.c[c], kp.c[c ^ 1], use_src, last);
        } else {
            k_pde<3><<<grid, 128, 0, st>>>(kp, kp.c[c], kp.c[c ^ 1], use_src, last);
        }
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

cudaError_t launch_init_positions(int dim, int periodic, const double *lo_d, const double *hi_d, uint64_t seed, int64_t n,
                                  int64_t n_alpha, float sigma_frac, float *pos, uint8_t *sp, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const float3 lo = make_float3((float)lo_d[0], (float)lo_d[1], (float)lo_d[2]);
    const float3 hi = make_float3((float)hi_d[0], (float)hi_d[1], (float)hi_d[2]);
    k_init_positions<<<blocks_for(n), TPB, 0, st>>>(dim, periodic, lo, hi, n, n_alpha, sigma_frac, (uint32_t)seed,
                                                    (uint32_t)(seed >> 32), pos, sp);
    return cudaGetLastError();
}

cudaError_t launch_stage_bins(const KP &kp, int32_t *cells, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    k_stage_bins<<<blocks_for(kp.n), TPB, 0, st>>>(kp, cells);
    return cudaGetLastError();
}

cudaError_t launch_stage_sort(const KP &kp, uint32_t *ids, uint32_t *bin_starts, cudaStream_t st)
{
    if (ids && kp.n > 0) k_stage_sort<<<blocks_for(kp.n), TPB, 0, st>>>(kp, ids);
    if (bin_starts) k_stage_starts<<<blocks_for(kp.bin_slots + 1), TPB, 0, st>>>(kp, bin_starts);
    return cudaGetLastError();
}

cudaError_t launch_stage_forces(const KP &kp, float *F, int32_t *count, unsigned long long *idsum, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    pair_kernel_attributes();
    const unsigned nb = blocks_for(kp.n);
#define STAGE_F(D, P, W) k_stage_forces<D, P, W><<<nb, TPB, pair_smem<D, P, W>(), st>>>(kp, F, count, idsum)
    const bool w = kp.search == 1;
    if (kp.dim == 2) {
        if (kp.periodic) w ? STAGE_F(2, true, true) : STAGE_F(2, true, false);
        else w ? STAGE_F(2, false, true) : STAGE_F(2, false, false);
    } else {
        if (kp.periodic) w ? STAGE_F(3, true, true) : STAGE_F(3, true, false);
        else w ? STAGE_F(3, false, true) : STAGE_F(3, false, false);
    }
#undef STAGE_F
    if (kp.pairs && kp.Fh) {
        // the forces of the half-window kernel replace the full window's
        // (the counts and id sums stay the full window's)
        if (kp.dim == 2) kp.periodic ? half_pairs_launch<2, true>(kp, st) : half_pairs_launch<2, false>(kp, st);
        else kp.periodic ? half_pairs_launch<3, true>(kp, st) : half_pairs_launch<3, false>(kp, st);
        if (kp.dim == 2) k_stage_take_half<2><<<nb, TPB, 0, st>>>(kp, F);
        else k_stage_take_half<3><<<nb, TPB, 0, st>>>(kp, F);
    }
    return cudaGetLastError();
}

cudaError_t launch_hard_sphere(const KP &kp, cudaStream_t st, int *launches)
{
    if (kp.n == 0) return cudaSuccess;
    const unsigned nb = blocks_for(kp.n * HS_TPC);
    if (kp.dim == 2) {
        if (kp.periodic) k_hard_sphere<2, true><<<nb, TPB, 0, st>>>(kp);
        else k_hard_sphere<2, false><<<nb, TPB, 0, st>>>(kp);
    } else {
        if (kp.periodic) k_hard_sphere<3, true><<<nb, TPB, 0, st>>>(kp);
        else k_hard_sphere<3, false><<<nb, TPB, 0, st>>>(kp);
    }
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_kde(const KP &kp, float *S, float *R, cudaStream_t st, int *launches)
{
    if (!kp.has_grid || kp.G == 0) return cudaSuccess;
    const unsigned nb = blocks_for(kp.G);
    if (kp.dim == 2) {
        if (kp.periodic) k_kde<2, true><<<nb, TPB, 0, st>>>(kp, S, R);
        else k_kde<2, false><<<nb, TPB, 0, st>>>(kp, S, R);
    } else {
        if (kp.periodic) k_kde<3, true><<<nb, TPB, 0, st>>>(kp, S, R);
        else k_kde<3, false><<<nb, TPB, 0, st>>>(kp, S, R);
    }
    if (launches) ++*launches;
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
