// slabs.cu -- kernels of the z-slab decomposition: ingest of exchanged cell
// records into a sub-domain, selection of a sub-domain's own cells for its
// neighbours and itself, and the addition of grid planes (the deposit on the
// halo planes folded into the owner's source).
//
// A record (chemo_cell of include/chemo.h) is two float4: (x, y, z, tag) and
// (dx, dy, dz, 0), tag = id | species << 29 with id ID_MASK for a ghost --
// the encoding of the state array's .w, so records move without re-packing.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include "chemo_internal.cuh"

namespace chemo {

namespace {

constexpr int STPB = 256;

unsigned blocks_of(int64_t n) { return (unsigned)((n + STPB - 1) / STPB); }

// k_pack_cells: records -> U (with their ids), counted into the next bins.
__global__ void __launch_bounds__(STPB) k_pack_cells(KP kp, const float4 *__restrict__ rec)
{
    const int64_t i = (int64_t)blockIdx.x * STPB + threadIdx.x;
    if (i >= kp.n) return;
    const float4 a = rec[2 * i], b = rec[2 * i + 1];
    float x[3] = {a.x, a.y, a.z};
    for (int q = 0; q < 3; ++q) {
        float v = x[q];
        if (!isfinite(v)) {
            set_err(kp, ERR_NONFINITE);
            v = kp.lo[q];
        }
        if (v < kp.lo[q] || v > kp.hi[q]) {
            set_err(kp, ERR_DOMAIN);
            v = fminf(fmaxf(v, kp.lo[q]), kp.hi[q]);
        }
        x[q] = v;
    }
    const uint32_t tag = __float_as_uint(a.w);
    uint32_t s = tag >> SP_SHIFT;
    if ((int)s >= kp.ns) {
        set_err(kp, ERR_SPECIES);
        s = 0;
    }
    const float4 u = make_float4(x[0], x[1], x[2], __uint_as_float((tag & ID_MASK) | (s << SP_SHIFT)));
    kp.U[i] = u;
    if (kp.dU) kp.dU[i] = make_float4(b.x, b.y, b.z, 0.f);
    kp.slot[i] = count_bin(kp.cnt_nxt, key_of(kp, u), kp.err);
}

// k_slab_select: every own (non-ghost) cell of the sorted state is appended to
// each target whose [z0, z1) holds it, as a ghost when it lies outside the
// target's [own0, own1). One atomic per warp and target for the slots.
__global__ void __launch_bounds__(STPB) k_slab_select(KP kp, SlabSelect t)
{
    const int64_t j = (int64_t)blockIdx.x * STPB + threadIdx.x;
    const bool valid = j < kp.n;
    const float4 me = valid ? kp.S[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t w = __float_as_uint(me.w);
    const bool own = valid && (w & ID_MASK) != ID_MASK;
    const float4 d = (own && kp.dS) ? kp.dS[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < t.nt; ++k) {
        const bool sel = own && me.z >= t.z0[k] && me.z < t.z1[k];
        const bool owned = sel && me.z >= t.own0[k] && me.z < t.own1[k];
        const unsigned m = __ballot_sync(0xffffffffu, sel);
        if (!m) continue;
        const unsigned mo = __ballot_sync(0xffffffffu, owned);
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0ull;
        if (lane == leader) {
            base = atomicAdd(&t.count[k][0], (unsigned long long)__popc(m));
            if (mo) atomicAdd(&t.count[k][1], (unsigned long long)__popc(mo));
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        if (sel) {
            const unsigned long long slot = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
            if (slot < (unsigned long long)t.cap[k]) {
                const uint32_t tag = owned ? w : (ID_MASK | (w & ~ID_MASK));
                t.out[k][2 * slot] = make_float4(me.x, me.y, me.z, __uint_as_float(tag));
                t.out[k][2 * slot + 1] = make_float4(d.x, d.y, d.z, 0.f);
            }
        }
    }
}

__global__ void __launch_bounds__(STPB) k_add(float *__restrict__ dst, const float *__restrict__ src, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * STPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * STPB)
        dst[i] += src[i];
}

}  // namespace

cudaError_t launch_pack_cells(const KP &kp, const float4 *rec, cudaStream_t st)
{
    if (kp.n == 0) return cudaSuccess;
    k_pack_cells<<<blocks_of(kp.n), STPB, 0, st>>>(kp, rec);
    return cudaGetLastError();
}

cudaError_t launch_slab_select(const KP &kp, const SlabSelect &t, cudaStream_t st)
{
    if (kp.n == 0 || t.nt == 0) return cudaSuccess;
    k_slab_select<<<blocks_of(kp.n), STPB, 0, st>>>(kp, t);
    return cudaGetLastError();
}

cudaError_t launch_add(float *dst, const float *src, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int64_t b = (n + STPB - 1) / STPB;
    k_add<<<(unsigned)(b < 4864 ? b : 4864), STPB, 0, st>>>(dst, src, n);
    return cudaGetLastError();
}

}  // namespace chemo
