// observe.cu -- device reductions of observables of the current state (the
// statistics of the paper's Sect. 4: cells per species, mean displacement and
// mean-square displacement per species; the chemical mass; occupancy
// histograms of the cells), so long runs report them without copying the
// state to the host. Per replicate for ensembles.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "chemo_engine.h"

using namespace chemo;

namespace {

constexpr int OTPB = 256;
constexpr int OBS_Q = 5;  // per species: count, sum dx, sum dy, sum dz, sum |d|^2

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums per (layer, species) into acc[layer][MAXS][OBS_Q]. A warp whose cells
// share a layer (the sorted state is layer-major) reduces with shuffles and
// adds once per species; a warp across two layers adds per cell.
__global__ void __launch_bounds__(OTPB) k_observe_cells(KP kp, double *__restrict__ acc)
{
    const int64_t stride = (int64_t)gridDim.x * OTPB;
    const int64_t nround = (kp.n + 31) / 32 * 32;  // every lane of a warp runs the same trips
    for (int64_t j = (int64_t)blockIdx.x * OTPB + threadIdx.x; j < nround; j += stride) {
        const bool valid = j < kp.n;
        float4 u = make_float4(0.f, 0.f, 0.f, 0.f), d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            u = kp.S[j];
            if (kp.dS) d = kp.dS[j];
        }
        const int sp = valid ? (int)(__float_as_uint(u.w) >> SP_SHIFT) : 0;
        const int lay = valid ? layer_of(kp, u) : 0;
        const float dz = kp.dim == 3 ? d.z : 0.f;
        const float q[OBS_Q] = {valid ? 1.f : 0.f, d.x, d.y, dz, d.x * d.x + d.y * d.y + dz * dz};
        const int lay0 = __shfl_sync(0xffffffffu, lay, 0);
        const bool uniform = __all_sync(0xffffffffu, !valid || lay == lay0);
        if (uniform) {
            for (int s = 0; s < kp.ns; ++s) {
                const bool mine = valid && sp == s;
                if (!__any_sync(0xffffffffu, mine)) continue;
#pragma unroll
                for (int k = 0; k < OBS_Q; ++k) {
                    const float v = warp_sum(mine ? q[k] : 0.f);
                    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[((int64_t)lay0 * MAXS + s) * OBS_Q + k], (double)v);
                }
            }
        } else if (valid) {
#pragma unroll
            for (int k = 0; k < OBS_Q; ++k) atomicAdd(&acc[((int64_t)lay * MAXS + sp) * OBS_Q + k], (double)q[k]);
        }
    }
}

// Chemical mass per layer, h^d sum_k tau_k c_k (trapezoid weights: 1/2 per
// wall axis at boundary nodes, 1 on a periodic grid), into mass[layer].
__global__ void __launch_bounds__(OTPB) k_observe_mass(KP kp, const float *__restrict__ c, double hd,
                                                       double *__restrict__ mass)
{
    const int gx = kp.g[0], gy = kp.g[1], gz = kp.dim == 3 ? kp.g[2] : 1;
    const int64_t plane = (int64_t)gx * gy * gz;  // nodes of one layer
    const int64_t stride = (int64_t)gridDim.x * OTPB;
    const int64_t nround = (kp.G + 31) / 32 * 32;
    const bool walls = kp.pde_bc != 2;
    for (int64_t g = (int64_t)blockIdx.x * OTPB + threadIdx.x; g < nround; g += stride) {
        float v = 0.f;
        int64_t lay = 0;
        if (g < kp.G) {
            lay = g / plane;
            const int64_t r = g - lay * plane;
            const int x = (int)(r % gx), y = (int)((r / gx) % gy), z = (int)(r / ((int64_t)gx * gy));
            float tau = 1.f;
            if (walls) {
                if (x == 0 || x == gx - 1) tau *= 0.5f;
                if (y == 0 || y == gy - 1) tau *= 0.5f;
                if (kp.dim == 3 && (z == 0 || z == gz - 1)) tau *= 0.5f;
            }
            v = tau * c[g];
        }
        const int64_t lay0 = __shfl_sync(0xffffffffu, lay, 0);
        if (__all_sync(0xffffffffu, g >= kp.G || lay == lay0)) {
            const float w = warp_sum(v);
            if ((threadIdx.x & 31) == 0) atomicAdd(&mass[lay0], (double)w * hd);
        } else if (g < kp.G) {
            atomicAdd(&mass[lay], (double)v * hd);
        }
    }
}

// Sums to the caller's layout: per layer MAXS x [count, mean dx, mean dy,
// mean dz, mean |d|^2] then the chemical mass.
__global__ void k_observe_finish(const double *__restrict__ acc, const double *__restrict__ mass, int layers,
                                 double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int per = MAXS * OBS_Q + 1;
    if (i >= layers * per) return;
    const int l = i / per, k = i - l * per;
    if (k == MAXS * OBS_Q) {
        out[i] = mass[l];
        return;
    }
    const int s = k / OBS_Q, q = k - s * OBS_Q;
    const double cnt = acc[((int64_t)l * MAXS + s) * OBS_Q];
    out[i] = q == 0 ? cnt : (cnt > 0.0 ? acc[((int64_t)l * MAXS + s) * OBS_Q + q] / cnt : 0.0);
}

// Occupancy histogram: hist[layer][species][bz][by][bx] += 1 per cell, the
// box cut into shape[a] equal parts per axis. Cells of a warp in the same
// histogram bin are added once (a match over the warp).
__global__ void __launch_bounds__(OTPB) k_histogram(KP kp, int hx, int hy, int hz, float *__restrict__ hist)
{
    const int64_t j = (int64_t)blockIdx.x * OTPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 u = kp.S[j];
    const int sp = (int)(__float_as_uint(u.w) >> SP_SHIFT);
    const int lay = layer_of(kp, u);
    const int hs[3] = {hx, hy, hz};
    const float pc[3] = {u.x, u.y, u.z};
    int64_t b = 0;
    for (int a = kp.dim - 1; a >= 0; --a) {
        const float f = (pc[a] - kp.lo[a]) / (kp.hi[a] - kp.lo[a]);
        int k = (int)floorf(f * (float)hs[a]);
        k = k < 0 ? 0 : (k >= hs[a] ? hs[a] - 1 : k);
        b = b * hs[a] + k;
    }
    const int64_t cells = (int64_t)hx * hy * (kp.dim == 3 ? hz : 1);
    const int64_t key = ((int64_t)lay * kp.ns + sp) * cells + b;
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, key);
    if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&hist[key], (float)__popc(same));
}

}  // namespace

extern "C" int chemo_observables(chemo_sim *s, double *out, int mem_kind, void *stream)
{
    ChemoRange nvtx_range("chemo_observables");
    if (s && s->kp.sub) return eng_fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_observables");
    if (!s || !out) return eng_fail(CHEMO_EINVAL, "sim and out are required");
    if (mem_kind != CHEMO_MEM_HOST && mem_kind != CHEMO_MEM_DEVICE) return eng_fail(CHEMO_EINVAL, "bad mem_kind");
    cudaStream_t st = (cudaStream_t)stream;
    const KP kp = eng_view(s);
    const int layers = std::max(kp.layers, 1);
    const int per = MAXS * OBS_Q + 1;
    const size_t nacc = (size_t)layers * MAXS * OBS_Q, nout = (size_t)layers * per;
    void *p;
    if (int r = eng_scratch(s, (nacc + (size_t)layers + nout) * sizeof(double) + 256, &p)) return r;
    double *acc = (double *)p, *mass = acc + nacc, *res = mass + layers;
    if (cudaMemsetAsync(acc, 0, (nacc + (size_t)layers) * sizeof(double), st) != cudaSuccess)
        return eng_fail(CHEMO_ECUDA, "chemo_observables: clearing the sums failed");
    if (kp.n > 0) {
        const unsigned nb = (unsigned)std::min<int64_t>((kp.n + OTPB - 1) / OTPB, 152 * 8);
        k_observe_cells<<<nb, OTPB, 0, st>>>(kp, acc);
    }
    if (kp.has_grid && kp.G > 0) {
        double hd = 1.0;
        for (int a = 0; a < kp.dim; ++a) hd *= kp.hgrid_d[a];
        const unsigned nb = (unsigned)std::min<int64_t>((kp.G + OTPB - 1) / OTPB, 152 * 8);
        k_observe_mass<<<nb, OTPB, 0, st>>>(kp, kp.c[s->cur], hd, mass);
    }
    k_observe_finish<<<(unsigned)((nout + 127) / 128), 128, 0, st>>>(acc, mass, layers, res);
    if (cudaGetLastError() != cudaSuccess) return eng_fail(CHEMO_ECUDA, "chemo_observables: launch failed");
    if (cudaMemcpyAsync(out, res, nout * sizeof(double),
                        mem_kind == CHEMO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
        return eng_fail(CHEMO_ECUDA, "chemo_observables: copy failed");
    if (mem_kind == CHEMO_MEM_HOST && cudaStreamSynchronize(st) != cudaSuccess)
        return eng_fail(CHEMO_ECUDA, "chemo_observables: synchronise failed");
    return CHEMO_OK;
}

extern "C" int chemo_histogram(chemo_sim *s, const int32_t *shape, float *hist_out, int mem_kind, void *stream)
{
    ChemoRange nvtx_range("chemo_histogram");
    if (s && s->kp.sub) return eng_fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_histogram");
    if (!s || !shape || !hist_out) return eng_fail(CHEMO_EINVAL, "sim, shape and hist_out are required");
    if (mem_kind != CHEMO_MEM_HOST && mem_kind != CHEMO_MEM_DEVICE) return eng_fail(CHEMO_EINVAL, "bad mem_kind");
    const KP kp = eng_view(s);
    const int hz = kp.dim == 3 ? shape[2] : 1;
    if (shape[0] < 1 || shape[1] < 1 || hz < 1 || shape[0] > 4096 || shape[1] > 4096 || hz > 4096)
        return eng_fail(CHEMO_EINVAL, "histogram shape must be 1..4096 per axis");
    const int64_t cells = (int64_t)shape[0] * shape[1] * hz;
    const int64_t total = (int64_t)std::max(kp.layers, 1) * kp.ns * cells;
    if (total > ((int64_t)1 << 28)) return eng_fail(CHEMO_EINVAL, "histogram too large");
    cudaStream_t st = (cudaStream_t)stream;
    void *p;
    if (int r = eng_scratch(s, (size_t)total * sizeof(float) + 256, &p)) return r;
    float *h = (float *)p;
    if (cudaMemsetAsync(h, 0, (size_t)total * sizeof(float), st) != cudaSuccess)
        return eng_fail(CHEMO_ECUDA, "chemo_histogram: clearing failed");
    if (kp.n > 0) k_histogram<<<(unsigned)((kp.n + OTPB - 1) / OTPB), OTPB, 0, st>>>(kp, shape[0], shape[1], hz, h);
    if (cudaGetLastError() != cudaSuccess) return eng_fail(CHEMO_ECUDA, "chemo_histogram: launch failed");
    if (cudaMemcpyAsync(hist_out, h, (size_t)total * sizeof(float),
                        mem_kind == CHEMO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
        return eng_fail(CHEMO_ECUDA, "chemo_histogram: copy failed");
    if (mem_kind == CHEMO_MEM_HOST && cudaStreamSynchronize(st) != cudaSuccess)
        return eng_fail(CHEMO_ECUDA, "chemo_histogram: synchronise failed");
    return CHEMO_OK;
}
