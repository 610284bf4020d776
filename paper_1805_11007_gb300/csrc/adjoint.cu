// adjoint.cu -- recording and vector-Jacobian product (adjoint) of the
// chemotaxis step (arXiv:1805.11007), for gradients of trajectory
// observables with respect to chi, the interaction strength and the
// diffusivities (parameter inference).
//
// One forward step maps (X^n, c^n) to (X^{n+1}, c^{n+1}):
//   Y_i      = X_i + dt (F_i(X) + chi_s G(X_i; c^n)) + sqrt(2 D_s dt) xi_i
//   X^{n+1}  = B(Y)                      (reflection or periodic wrap)
//   c^{n+1}  = PDE substeps of c^n with the source S(X^{n+1})
// with the noise xi frozen (the Philox counter is the step index). The
// reverse sweep, for n = N-1 .. 0, given lambda_X = dL/dX^{n+1} and
// lambda_c = dL/dc^{n+1}:
//   1. PDE transpose: mu <- mu + dt_s (D_c Lap^T mu - gamma mu) per substep,
//      accumulating lambda_S = sum over substeps of mu / s;
//   2. deposit transpose: lambda_X_i += k_s dt/h^d sum_k lambda_S[k]/tau_k grad w_k(X^{n+1}_i);
//   3. boundary: lambda_Y = J_B^T lambda_X (a sign per reflection);
//   4. lambda_X^n = lambda_Y + dt chi_s (dG/dX)^T lambda_Y
//                   + dt sum_j H_ij (lambda_Y_i - lambda_Y_j),
//      H = f/r (I - d d^T) + f'(r) d d^T (pair force Jacobian, symmetric);
//      lambda_c^n = mu^(0) + dt chi_s (dG/dc)^T lambda_Y (scatter to the nodes);
//   5. parameters: dL/dchi += dt chemotactic_s G . lambda_Y,
//      dL/dinter += dt (F/inter) . lambda_Y, dL/dD_s += sqrt(dt/(2 D_s)) xi . lambda_Y.
// The cutoff jump and the reflection kinks are measure-zero events and are
// not differentiated.
//
// Memory: checkpoints of (X, c) every `every` steps; each segment is re-run
// forward to store its states before its reverse sweep. The re-run of segment
// s - 1 (one stream, the simulation's buffers) overlaps the reverse sweep of
// segment s (a second stream, the tape's buffers), with two segment buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "chemo_engine.h"

using namespace chemo;

namespace {

constexpr int ATPB = 128;  // small blocks: the adjoint kernels run over tens of thousands of cells

// States of one segment, stored by its forward re-run for its reverse sweep.
struct SegBuf {
    float *pos = nullptr;     // (every + 1) x n x dim, by id
    float *c = nullptr;       // every x G
    float4 *S = nullptr;      // sorted state at the start of each step
    uint32_t *cnt = nullptr;  // its bin counts (packed 16-bit)
    uint32_t *gst = nullptr;  // its group offsets
    float *F = nullptr;       // pair force of each step, by id (n x dim)
};

struct Tape {
    int64_t n = 0, G = 0, nsteps = 0, every = 0, step0 = 0;
    int nseg = 0, dim = 0, ns = 0;
    DevMem mem;  // the simulation's allocator
    std::vector<DevBuf> allocs;
    std::vector<float *> ck_pos, ck_c;  // checkpoints: positions by id (n x dim), field
    uint8_t *species = nullptr;         // species by id
    uint16_t *layer_id = nullptr;       // replicate of each id (NULL for a single simulation)
    // two segment buffers: segment s - 1 is re-run into one while the
    // reverse sweep of segment s reads the other (two streams)
    SegBuf sb[2];
    SegBuf sb_all;  // the block behind sb[0], sb[1] (2 every steps, 2 (every + 1) position slots)
    // segments whose states the recorded run stored (pos == NULL: re-run)
    std::vector<SegBuf> stored;
    cudaStream_t s_fwd = nullptr, s_rev = nullptr;
    cudaStream_t s_pair = nullptr;  // pair term of step k beside the PDE transpose of step k - 1
    cudaEvent_t ev_cells = nullptr, ev_pairs = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr, ev_fwd_end = nullptr, ev_rev_end = nullptr;
    float *lamX[2] = {nullptr, nullptr};  // n x dim by id
    float *lamY = nullptr;              // n x dim by id
    float *lamC[2] = {nullptr, nullptr};  // G
    float *lamS = nullptr;              // G
    size_t cwords = 0, gwords = 0;      // words of one count table / offset table
    float *dpf = nullptr;               // parameter gradient (float) for the caller
    double *dpar = nullptr;             // (2 + MAXS) x pstride per-block partials
    int64_t pstride = 0;                // blocks of the per-cell kernel
};

}  // namespace

struct chemo_tape : Tape {};

void chemo_tape_free(chemo_tape *t)
{
    if (!t) return;
    if (t->s_fwd) cudaStreamSynchronize(t->s_fwd);
    if (t->s_rev) cudaStreamSynchronize(t->s_rev);
    if (t->s_pair) cudaStreamSynchronize(t->s_pair);
    // cudaFree waits for the device by itself; a caller's release does not,
    // and the record may have run on the caller's stream
    if (t->mem.release && !t->allocs.empty()) cudaDeviceSynchronize();
    for (const DevBuf &b : t->allocs) eng_mem_release(t->mem, b.ptr, b.bytes);
    for (cudaEvent_t e : {t->ev_ready[0], t->ev_ready[1], t->ev_done[0], t->ev_done[1], t->ev_start, t->ev_fwd_end,
                          t->ev_rev_end, t->ev_cells, t->ev_pairs})
        if (e) cudaEventDestroy(e);
    if (t->s_fwd) cudaStreamDestroy(t->s_fwd);
    if (t->s_rev) cudaStreamDestroy(t->s_rev);
    if (t->s_pair) cudaStreamDestroy(t->s_pair);
    delete t;
}

namespace {

int talloc(chemo_tape *t, void **p, size_t bytes)
{
    size_t b = 0;
    if (int r = eng_mem_alloc(t->mem, p, bytes, &b)) return r;
    t->allocs.push_back({*p, b});
    return CHEMO_OK;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Positions (n x dim) and species of the sorted state, by id.
__global__ void k_gather_state(KP kp, float *__restrict__ pos, uint8_t *__restrict__ sp)
{
    const int64_t j = (int64_t)blockIdx.x * ATPB + threadIdx.x;
    if (j >= kp.n) return;
    const float4 u = kp.S[j];
    const uint32_t w = __float_as_uint(u.w);
    const int64_t id = gid_of(kp, u);  // replicates: the layer's offset plus the id within it
    if (id >= kp.n) return;
    pos[id * kp.dim + 0] = u.x;
    pos[id * kp.dim + 1] = u.y;
    if (kp.dim == 3) pos[id * kp.dim + 2] = u.z;
    if (sp) sp[id] = (uint8_t)(w >> SP_SHIFT);
}

// Transposed Laplacian along one axis at node k (N nodes, stride): with
// mirror ghosts the wall rows are (-2, 2) so the transpose differs there.
__device__ __forceinline__ float lapT_axis(const float *__restrict__ mu, int64_t g, int k, int N, int64_t stride,
                                           bool periodic)
{
    const float m0 = mu[g];
    if (periodic) {
        const int64_t gl = k > 0 ? g - stride : g + (int64_t)(N - 1) * stride;
        const int64_t gr = k < N - 1 ? g + stride : g - (int64_t)(N - 1) * stride;
        return mu[gl] + mu[gr] - 2.f * m0;
    }
    const float left = k == 0 ? 0.f : (k == 1 ? 2.f * mu[g - stride] : mu[g - stride]);
    const float right = k == N - 1 ? 0.f : (k == N - 2 ? 2.f * mu[g + stride] : mu[g + stride]);
    return left + right - 2.f * m0;
}

// One transposed PDE substep: mu_out = mu_in + dt_s (D_c Lap^T - gamma) mu_in,
// lamS (+)= mu_in / s.
__global__ void k_adj_pde(KP kp, const float *__restrict__ mu_in, float *__restrict__ mu_out, float *__restrict__ lamS,
                          float inv_s, int first)
{
    const int64_t g = (int64_t)blockIdx.x * ATPB + threadIdx.x;
    if (g >= kp.G) return;
    const int gx = kp.g[0], gy = kp.g[1];
    const int x = (int)(g % gx);
    const int y = (int)((g / gx) % gy);
    const int z = kp.dim == 3 ? (int)(g / ((int64_t)gx * gy)) : 0;
    const bool per = kp.pde_bc == 2;
    float lap = lapT_axis(mu_in, g, x, gx, 1, per) * kp.inv_h2[0] + lapT_axis(mu_in, g, y, gy, gx, per) * kp.inv_h2[1];
    if (kp.dim == 3) lap += lapT_axis(mu_in, g, z, kp.g[2], (int64_t)gx * gy, per) * kp.inv_h2[2];
    const float m = mu_in[g];
    mu_out[g] = m + kp.dts * (kp.Dc * lap - kp.gamma * m);
    lamS[g] = (first ? 0.f : lamS[g]) + m * inv_s;
}

__device__ __forceinline__ int64_t nidx(const KP &kp, const int *k) { return gidx(kp, k[0], k[1], k[2]); }

// Grid cell of x per axis (lower and upper node, offset in the cell).
template <int DIM>
__device__ __forceinline__ void cell_frac(const KP &kp, const float *x, int k0[3], int k1[3], float f[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        k0[a] = k1[a] = 0;
        f[a] = 0.f;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) gcell(kp, a, x[a], k0[a], k1[a], f[a]);
}

// Corner m of the 2^d nodes of a grid cell: node indices, multilinear
// weight and its gradient d(weight)/dx_b.
template <int DIM>
__device__ __forceinline__ void corner_w(const KP &kp, const int k0[3], const int k1[3], const float f[3], int m,
                                         int node[3], float &w, float dw[3])
{
    w = 1.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int bit = (m >> a) & 1;
        node[a] = a < DIM ? (bit ? k1[a] : k0[a]) : k0[a];  // beyond DIM: the replicate's layer
        if (a < DIM) w *= bit ? f[a] : 1.f - f[a];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float d = 0.f;
        if (b < DIM) {
            d = ((m >> b) & 1) ? kp.inv_h[b] : -kp.inv_h[b];
#pragma unroll
            for (int a = 0; a < DIM; ++a)
                if (a != b) d *= ((m >> a) & 1) ? f[a] : 1.f - f[a];
        }
        dw[b] = d;
    }
}

// Sum over the NC consecutive lanes of a cell's group (NC divides 32).
template <int NC>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = 1; o < NC; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-cell adjoint terms (by id), 2^d threads per cell: thread m of a cell's
// group takes grid corner m of the deposit transpose at X^{n+1}, of the
// gradient interpolation at X^n with its Jacobian, and of the interpolation
// transpose; the group adds the corners' parts with shuffles (one thread per
// cell left the adjoint's per-cell kernel latency bound at a few warps per
// SM). Reads X^n, X^{n+1}, c^n, lambda_X^{n+1}, lambda_S and the step's pair
// force Fb (f_unit Fb = dF/dinter); writes lambda_Y and the local part of
// lambda_X^n, scatters the interpolation transpose into lambda_c and adds
// the parameter gradients to the block's slots of dpar (launched over
// n 2^d threads).
template <int DIM>
__global__ void __launch_bounds__(ATPB) k_adj_cells(KP kp, const float *__restrict__ Xn, const float *__restrict__ Xn1,
                                                    const uint8_t *__restrict__ spec, const float *__restrict__ cn,
                                                    const float *__restrict__ lamX1, const float *__restrict__ lamS,
                                                    const float *__restrict__ Fb, float f_unit, float *__restrict__ lamY,
                                                    float *__restrict__ lamXn, float *__restrict__ lamC,
                                                    unsigned long long step, double *dpar, int64_t pstride,
                                                    int has_grid, int lams_over_tau,
                                                    const uint16_t *__restrict__ layer_id)
{
    constexpr int NC = 1 << DIM;
    static_assert(32 % NC == 0 && ATPB % 32 == 0, "a cell's threads lie in one warp");
    __shared__ float red[ATPB / 32][2 + MAXS];
    const int64_t t = (int64_t)blockIdx.x * ATPB + threadIdx.x;
    const int64_t i = t / NC;
    const int m = (int)(t % NC);
    const bool valid = i < kp.n;
    const int sp = valid ? (int)spec[i] : 0;
    // replicates (2D layers): the cell's layer is the third grid index and
    // keys its noise with its id within the layer
    const int layer = (valid && layer_id) ? (int)layer_id[i] : 0;
    const uint32_t lid = (uint32_t)(layer_id && valid ? i - kp.layer_off[layer] : i);
    float x0[3] = {0.f, 0.f, 0.f}, x1[3] = {0.f, 0.f, 0.f}, lx[3] = {0.f, 0.f, 0.f};
    if (valid)
        for (int a = 0; a < DIM; ++a) {
            x0[a] = Xn[i * DIM + a];
            x1[a] = Xn1[i * DIM + a];
            lx[a] = lamX1[i * DIM + a];
        }
    // 2. deposit transpose at X^{n+1}: this corner's part
    float dl[3] = {0.f, 0.f, 0.f};
    if (valid && has_grid && kp.src[sp] != 0.f) {
        int k0[3], k1[3], nd[3];
        float f[3], wm, dwm[3];
        cell_frac<DIM>(kp, x1, k0, k1, f);
        if (DIM == 2) k0[2] = k1[2] = layer;
        corner_w<DIM>(kp, k0, k1, f, m, nd, wm, dwm);
        float inv_tau = 1.f;
        if (kp.pde_bc != 2 && !lams_over_tau)  // (already divided by tau when lams_over_tau)
            for (int a = 0; a < DIM; ++a)
                if (nd[a] == 0 || nd[a] == kp.g[a] - 1) inv_tau *= 2.f;
        const float l = lamS[nidx(kp, nd)] * inv_tau * kp.src[sp];
        for (int a = 0; a < DIM; ++a) dl[a] = l * dwm[a];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) lx[a] += group_sum<NC>(dl[a]);
    // forward quantities at X^n: gradient interpolation and its Jacobian
    const float chem = kp.chem[sp];
    float G[3] = {0.f, 0.f, 0.f}, J[3][3] = {{0.f}};
    const bool interp = has_grid && kp.chem_mode == 0;
    int nd0[3] = {0, 0, 0};
    float w0 = 0.f;
    if (kp.chem_mode == 1) {
        for (int a = 0; a < DIM; ++a) G[a] = kp.fixed_g[a];
    } else if (interp) {
        if (valid) {
            int k0[3], k1[3];
            float f[3], dw0[3];
            cell_frac<DIM>(kp, x0, k0, k1, f);
            if (DIM == 2) k0[2] = k1[2] = layer;
            corner_w<DIM>(kp, k0, k1, f, m, nd0, w0, dw0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                int kp1[3] = {nd0[0], nd0[1], nd0[2]}, km1[3] = {nd0[0], nd0[1], nd0[2]};
                kp1[a] = gnbr(kp, a, nd0[a] + 1);
                km1[a] = gnbr(kp, a, nd0[a] - 1);
                const float ga = (cn[nidx(kp, kp1)] - cn[nidx(kp, km1)]) * kp.inv_2h[a];
                G[a] = w0 * ga;
#pragma unroll
                for (int b = 0; b < DIM; ++b) J[a][b] = dw0[b] * ga;
            }
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            G[a] = group_sum<NC>(G[a]);
#pragma unroll
            for (int b = 0; b < DIM; ++b) J[a][b] = group_sum<NC>(J[a][b]);
        }
    }
    float p_chi = 0.f, p_int = 0.f, p_Ds = 0.f;
    if (valid) {
        // noise and the pre-boundary position Y (reflection signs), in every
        // thread of the group
        const uint4 rw = cell_words(kp, lid, step, TAG_MOVE, (uint32_t)layer);
        const float2 n01 = box_muller(rw.x, rw.y);
        const float xi[3] = {n01.x, n01.y, DIM == 3 ? box_muller(rw.z, rw.w).x : 0.f};
        const float amp = kp.noise[sp];
        float sgn[3] = {1.f, 1.f, 1.f};
        for (int a = 0; a < DIM; ++a) {
            float y = x0[a] + kp.dt * (Fb[i * DIM + a] + chem * G[a]) + amp * xi[a];
            if (!kp.periodic) {
                for (int it = 0; it < 16 && (y < kp.lo[a] || y > kp.hi[a]); ++it) {
                    y = y < kp.lo[a] ? 2.f * kp.lo[a] - y : 2.f * kp.hi[a] - y;
                    sgn[a] = -sgn[a];
                }
            }
        }
        // 3. boundary, 4. local terms (thread a of the group writes axis a)
        float ly[3] = {0.f, 0.f, 0.f}, tx[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < DIM; ++a) ly[a] = sgn[a] * lx[a];
        for (int b = 0; b < DIM; ++b) {
            float tb = ly[b];
            if (interp && chem != 0.f) {
                float sj = 0.f;
                for (int a = 0; a < DIM; ++a) sj = fmaf(ly[a], J[a][b], sj);
                tb = fmaf(kp.dt * chem, sj, tb);
            }
            tx[b] = tb;
        }
        if (m < DIM) {
            lamY[i * DIM + m] = m == 0 ? ly[0] : (m == 1 ? ly[1] : ly[2]);
            lamXn[i * DIM + m] = m == 0 ? tx[0] : (m == 1 ? tx[1] : tx[2]);
        }
        // interpolation transpose onto the nodes: this corner
        if (interp && chem != 0.f) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const float coef = kp.dt * chem * w0 * ly[a] * kp.inv_2h[a];
                if (coef == 0.f) continue;
                int kp1[3] = {nd0[0], nd0[1], nd0[2]}, km1[3] = {nd0[0], nd0[1], nd0[2]};
                kp1[a] = gnbr(kp, a, nd0[a] + 1);
                km1[a] = gnbr(kp, a, nd0[a] - 1);
                atomicAdd(&lamC[nidx(kp, kp1)], coef);
                atomicAdd(&lamC[nidx(kp, km1)], -coef);
            }
        }
        // 5. parameters (the group's first thread)
        if (m == 0) {
            float gl = 0.f, fl = 0.f, xl = 0.f;
            for (int a = 0; a < DIM; ++a) {
                gl = fmaf(G[a], ly[a], gl);
                fl = fmaf(Fb[i * DIM + a] * f_unit, ly[a], fl);
                xl = fmaf(xi[a], ly[a], xl);
            }
            p_chi = kp.dt * kp.chemotactic_f[sp] * gl;
            p_int = kp.dt * fl;
            if (amp > 0.f) p_Ds = kp.dt / amp * xl;  // d sqrt(2 D dt)/dD = dt / sqrt(2 D dt)
        }
    }
    // parameter partials: each warp sums its cells' parts, the block adds the
    // warps' sums in double into its slot blockIdx.x of each parameter's row
    // (no two blocks share a slot and successive kernels run in order)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int np = 2 + kp.ns;
    for (int v = 0; v < np; ++v) {
        float x = v == 0 ? p_chi : (v == 1 ? p_int : (sp == v - 2 ? p_Ds : 0.f));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[wid][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < np) {
        double sum = 0.0;
        for (int w = 0; w < ATPB / 32; ++w) sum += (double)red[w][threadIdx.x];
        dpar[(int64_t)threadIdx.x * pstride + blockIdx.x] += sum;
    }
}

// Pair term of the adjoint over the cell list of X^n (sorted S):
// lambda_X^n_i += dt sum_j H_ij (lambda_Y_i - lambda_Y_j). APC threads share
// a cell (each takes every APC-th candidate of each row range) and sum their
// parts with shuffles. H_ij = f/r (I - d d^T) + f' d d^T is even in the
// difference d = X_i - X_j, so the term of j is the negation of the term of
// i: with HALF (walls), each pair is found once, by the cell whose upper
// half window holds the other (the rows at (dz, dy) > (0, 0) with all their
// bins, in its own row the next bin and the cells of its own bin after it),
// which adds the term to itself and its negation to the partner (float
// atomics, so the order of the additions is open); else every cell searches
// its whole window and adds its own term.
constexpr int APC = 8;

template <int DIM, bool PERIODIC, bool HALF>
__global__ void __launch_bounds__(ATPB) k_adj_pairs(KP kp, const float *__restrict__ lamY, float *__restrict__ lamXn)
{
    static_assert(!(HALF && PERIODIC), "the half window is taken with walls only");
    const int64_t t = (int64_t)blockIdx.x * ATPB + threadIdx.x;
    const int64_t j = t / APC;
    const int sub = (int)(t % APC);
    float acc[3] = {0.f, 0.f, 0.f};
    int64_t id = -1;
    if (j < kp.n) {
        id = gid_of(kp, kp.S[j]);  // replicates: the layer's offset plus the id within it
        if (id >= kp.n) id = -1;
    }
    if (id >= 0) {
        const float4 me = kp.S[j];
        const int sp = (int)(__float_as_uint(me.w) >> SP_SHIFT);
        float li[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < DIM; ++a) li[a] = lamY[id * DIM + a];
        int c[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        const float pc[3] = {me.x, me.y, me.z};
        for (int a = 0; a < DIM; ++a) {
            c[a] = bin_axis(pc[a], kp.lo[a], kp.inv_b[a], kp.nb[a]);
            const float f = __fmul_rn(__fsub_rn(pc[a], kp.lo[a]), kp.inv_b[a]) - (float)c[a];
            if (kp.search == 2) {
                lo[a] = f < 0.5f ? c[a] - 1 : c[a];
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
        if (DIM == 2) c[2] = lo[2] = hi[2] = layer_of(kp, me);  // the rows of the cell's own layer
        const uint32_t n = (uint32_t)kp.n;
        // one candidate: the pair term, added to this cell (and, with the
        // half window, its negation to the partner)
        auto term = [&](uint32_t q) {
            const float4 o = __ldg(&kp.S[q]);
            float d[3] = {me.x - o.x, me.y - o.y, DIM == 3 ? me.z - o.z : 0.f};
            if (PERIODIC)
                for (int a = 0; a < DIM; ++a) {
                    if (d[a] > kp.halfL[a]) d[a] -= kp.L[a];
                    else if (d[a] < -kp.halfL[a]) d[a] += kp.L[a];
                }
            const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            const int st = sp * MAXS + (int)(__float_as_uint(o.w) >> SP_SHIFT);
            if (!(r2 < kp.rc2[st]) || !(r2 > 0.f)) return;
            const int64_t jd = gid_of(kp, o);
            if (jd >= kp.n) return;
            const float r = sqrtf(r2), rinv = 1.f / r;
            const float e = __expf(-r * kp.inv_eps[st]);
            const float f = kp.amp_f[st] * (e - kp.shift[st]);
            const float fp = -kp.amp_f[st] * kp.inv_eps[st] * e;
            float dl[3], dot = 0.f;
            for (int a = 0; a < DIM; ++a) {
                dl[a] = li[a] - lamY[jd * DIM + a];
                dot = fmaf(d[a] * rinv, dl[a], dot);
            }
            const float s1 = f * rinv, s2 = (fp - f * rinv) * dot;
            for (int a = 0; a < DIM; ++a) {
                const float v = s1 * dl[a] + s2 * d[a] * rinv;
                acc[a] += v;
                if (HALF) atomicAdd(&lamXn[jd * DIM + a], -kp.dt * v);
            }
        };
        if (HALF) {
            // rows (oy, oz) of the upper half: the own row (0, 0), then (1, 0),
            // then (-1..1, 1) in 3D
            constexpr int NROWS = DIM == 3 ? 5 : 2;
            for (int k = 0; k < NROWS; ++k) {
                const int oy = k == 0 ? 0 : (k == 1 ? 1 : k - 3);
                const int oz = k < 2 ? 0 : 1;
                const int y = c[1] + oy, z = c[2] + oz;
                if (y < 0 || y >= kp.nb[1] || (DIM == 3 && z >= kp.nb[2])) continue;
                const uint32_t rowk = (uint32_t)kp.px * ((uint32_t)y + (uint32_t)kp.nb[1] * (uint32_t)z);
                const int x0 = max(k == 0 ? c[0] : c[0] - 1, 0), x1 = min(c[0] + 1, kp.nb[0] - 1);
                const uint32_t q0 = k == 0 ? (uint32_t)j + 1u : min(bin_start(kp.cnt_cur, kp.gstart, rowk + (uint32_t)x0), n);
                const uint32_t q1 = min(bin_start(kp.cnt_cur, kp.gstart, rowk + (uint32_t)x1 + 1u), n);
                for (uint32_t q = q0 + (uint32_t)sub; q < q1; q += APC) term(q);
            }
        } else {
            for (int z = lo[2]; z <= hi[2]; ++z) {
                int zz = z;
                if (PERIODIC && DIM == 3) zz = z < 0 ? z + kp.nb[2] : (z >= kp.nb[2] ? z - kp.nb[2] : z);
                for (int y = lo[1]; y <= hi[1]; ++y) {
                    int yy = y;
                    if (PERIODIC) yy = y < 0 ? y + kp.nb[1] : (y >= kp.nb[1] ? y - kp.nb[1] : y);
                    const uint32_t rowk = (uint32_t)kp.px * ((uint32_t)yy + (uint32_t)kp.nb[1] * (uint32_t)zz);
                    // the row's bins as contiguous ranges of the sorted array (a
                    // periodic row that wraps is two ranges)
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
                        for (uint32_t q = q0 + (uint32_t)sub; q < q1; q += APC)
                            if (q != (uint32_t)j) term(q);
                    }
                }
            }
        }
    }
    // the APC threads of a cell are consecutive lanes of one warp
    for (int o = APC / 2; o > 0; o >>= 1)
        for (int a = 0; a < DIM; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if (id >= 0 && sub == 0)
        for (int a = 0; a < DIM; ++a) {
            if (HALF) atomicAdd(&lamXn[id * DIM + a], kp.dt * acc[a]);  // partners add here too
            else lamXn[id * DIM + a] += kp.dt * acc[a];
        }
}

// Sums each parameter's row of per-block partials (one warp per parameter).
__global__ void k_params_out(const double *dpar, int64_t pstride, float *out, int np)
{
    const int p = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (p >= np) return;
    double s = 0.0;
    for (int64_t b = lane; b < pstride; b += 32) s += dpar[p * pstride + b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[p] = (float)s;
}

unsigned blocks(int64_t n) { return (unsigned)((n + ATPB - 1) / ATPB); }

#define ATRY(expr)                                                                                      \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return eng_fail(CHEMO_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

int check_adjoint_model(const chemo_sim *s)
{
    const chemo_params &p = s->prm;
    if (p.reactions) return eng_fail(CHEMO_ENOTSUP, "the adjoint does not cover type switching (reactions = 1)");
    if (p.move_scheme || p.hard_sphere || p.deposit_kernel)
        return eng_fail(CHEMO_ENOTSUP, "the adjoint covers the Euler-Maruyama move with the CIC deposit only");
    for (int i = 0; i < p.n_species; ++i)
        if (p.consume[i] != 0.f) return eng_fail(CHEMO_ENOTSUP, "the adjoint does not cover consumption (consume != 0)");
    if (p.chem_mode == 0 && p.pde_bc == 1) return eng_fail(CHEMO_ENOTSUP, "the adjoint does not cover Dirichlet walls");
    return CHEMO_OK;
}

// Current sorted state into (pos by id, species by id).
int gather(chemo_sim *s, float *pos, uint8_t *sp, cudaStream_t st)
{
    if (s->kp.n == 0) return CHEMO_OK;
    k_gather_state<<<blocks(s->kp.n), ATPB, 0, st>>>(eng_view(s), pos, sp);
    ATRY(cudaGetLastError());
    return CHEMO_OK;
}

float *cur_field(chemo_sim *s) { return s->kp.has_grid ? s->kp.c[s->cur] : nullptr; }

}  // namespace

namespace {

// Device memory of one segment's stored states.
size_t segment_bytes(const chemo_tape *t)
{
    const size_t E = (size_t)t->every, n1 = (size_t)std::max<int64_t>(t->n, 1);
    const size_t pb = n1 * t->dim * sizeof(float), gb = (size_t)std::max<int64_t>(t->G, 1) * sizeof(float);
    return pb * (E + 1) + gb * E + E * n1 * sizeof(float4) + E * (t->cwords + t->gwords) * sizeof(uint32_t) + E * pb +
           6 * 256;
}

// Buffers for the stored states of E steps (E + 1 position slots).
int alloc_steps(chemo_tape *t, SegBuf &B, size_t E)
{
    const size_t n1 = (size_t)std::max<int64_t>(t->n, 1);
    const size_t pb = n1 * t->dim * sizeof(float), gb = (size_t)std::max<int64_t>(t->G, 1) * sizeof(float);
    void *p;
    int r;
    if ((r = talloc(t, &p, pb * (E + 1)))) return r;
    B.pos = (float *)p;
    if ((r = talloc(t, &p, gb * E))) return r;
    B.c = (float *)p;
    if ((r = talloc(t, &p, E * n1 * sizeof(float4)))) return r;
    B.S = (float4 *)p;
    if ((r = talloc(t, &p, E * t->cwords * sizeof(uint32_t)))) return r;
    B.cnt = (uint32_t *)p;
    if ((r = talloc(t, &p, E * t->gwords * sizeof(uint32_t)))) return r;
    B.gst = (uint32_t *)p;
    if ((r = talloc(t, &p, E * pb))) return r;
    B.F = (float *)p;
    return CHEMO_OK;
}

// Points the particle kernel's tape at B for the steps step0 .. step0 + len - 1:
// each of those steps writes the positions before it, the field, the sorted
// state with its cell list and the pair force.
void set_tape(chemo_sim *s, const chemo_tape *t, const SegBuf &B, int64_t step0, int64_t len)
{
    KP::TapeOut &tp = s->kp.tape;
    tp = KP::TapeOut{};
    tp.pos = B.pos;
    tp.c = B.c;
    tp.F = B.F;
    tp.S = B.S;
    tp.cnt = B.cnt;
    tp.gst = B.gst;
    tp.s0 = (unsigned long long)step0;
    tp.nk = (unsigned long long)len;
    tp.cwords = (int64_t)t->cwords;
    tp.gwords = (int64_t)t->gwords;
}


}  // namespace

extern "C" int chemo_record(chemo_sim *s, int64_t nsteps, int32_t every, void *stream)
{
    return chemo_record_stored(s, nsteps, every, 0, stream);
}

extern "C" int chemo_record_stored(chemo_sim *s, int64_t nsteps, int32_t every, int64_t store_bytes, void *stream)
{
    ChemoRange nvtx_range("chemo_record_stored");
    if (s && s->kp.sub) return eng_fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_record_stored");
    if (!s || nsteps < 0 || every < 1) return eng_fail(CHEMO_EINVAL, "chemo_record: bad arguments");
    if (int r = check_adjoint_model(s)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    chemo_tape_free(s->tape);
    s->tape = new (std::nothrow) chemo_tape();
    if (!s->tape) return eng_fail(CHEMO_ENOMEM, "host allocation failed");
    chemo_tape *t = s->tape;
    t->mem = s->mem;
    const KP &kp = s->kp;
    t->n = kp.n;
    t->G = kp.has_grid ? kp.G : 0;
    t->nsteps = nsteps;
    t->every = every;
    t->step0 = s->step;
    t->dim = kp.dim;
    t->ns = kp.ns;
    t->nseg = (int)((nsteps + every - 1) / every);
    t->cwords = (size_t)kp.bin_slots / 2;
    t->gwords = ((size_t)kp.ngroups + 1 + 3) & ~(size_t)3;
    // the latest segments whose states fit in store_bytes are stored now
    // and not re-run by the gradient (the reverse sweep starts with them)
    const size_t sbytes = segment_bytes(t);
    const int64_t nstore = store_bytes < 0 ? t->nseg : std::min<int64_t>(t->nseg, store_bytes / (int64_t)sbytes);
    t->stored.assign((size_t)t->nseg, SegBuf{});
    const size_t pb = (size_t)std::max<int64_t>(t->n, 1) * kp.dim * sizeof(float);
    const size_t gb = (size_t)std::max<int64_t>(t->G, 1) * sizeof(float);
    void *p;
    int r;
    for (int k = 0; k <= t->nseg; ++k) {
        if ((r = talloc(t, &p, pb))) return r;
        t->ck_pos.push_back((float *)p);
        if ((r = talloc(t, &p, gb))) return r;
        t->ck_c.push_back((float *)p);
    }
    if ((r = talloc(t, &p, (size_t)std::max<int64_t>(t->n, 1)))) return r;
    t->species = (uint8_t *)p;
    if (kp.layers > 1 && t->n > 0) {  // replicates: the layer of every id, for the reverse sweep
        std::vector<uint16_t> lid((size_t)t->n);
        for (int l = 0; l < kp.layers; ++l)
            for (int64_t i = s->layer_off_host[(size_t)l]; i < s->layer_off_host[(size_t)l + 1]; ++i)
                lid[(size_t)i] = (uint16_t)l;
        if ((r = talloc(t, &p, (size_t)t->n * sizeof(uint16_t)))) return r;
        t->layer_id = (uint16_t *)p;
        if (cudaMemcpy(t->layer_id, lid.data(), lid.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess)
            return eng_fail(CHEMO_ECUDA, "chemo_record: layer table copy failed");
    }
    // the stored segments are the last nstore: steps k0 .. nsteps - 1 of the
    // run, kept in one block; each stored segment is a view into it
    const int fs = t->nseg - (int)nstore;
    const int64_t k0 = (int64_t)fs * every, nk = nsteps - k0;
    SegBuf all{};
    if (nstore > 0) {
        if ((r = alloc_steps(t, all, (size_t)nk))) return r;
        const size_t n1 = (size_t)std::max<int64_t>(t->n, 1), g1 = (size_t)std::max<int64_t>(t->G, 1);
        for (int k = fs; k < t->nseg; ++k) {
            const size_t o = (size_t)((int64_t)k * every - k0);
            SegBuf &B = t->stored[(size_t)k];
            B.pos = all.pos + o * n1 * t->dim;
            B.c = all.c + o * g1;
            B.S = all.S + o * n1;
            B.cnt = all.cnt + o * t->cwords;
            B.gst = all.gst + o * t->gwords;
            B.F = all.F + o * n1 * t->dim;
        }
    }
    // forward with checkpoints at the start of every segment and at the end;
    // over the stored steps the particle kernel writes the tape (indexed by
    // the device's step counter, so the graphs of chemo_step_n replay it:
    // they are captured afresh with the tape set and dropped after)
    int rc = CHEMO_OK;
    for (int k = 0; k <= t->nseg && rc == CHEMO_OK; ++k) {
        if ((rc = gather(s, t->ck_pos[k], k == 0 ? t->species : nullptr, st))) break;
        if (t->G && cudaMemcpyAsync(t->ck_c[k], cur_field(s), gb, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            rc = eng_fail(CHEMO_ECUDA, "chemo_record: checkpoint copy failed");
            break;
        }
        if (k == t->nseg) break;
        if (k == fs) {
            eng_drop_graphs(s);
            set_tape(s, t, all, t->step0 + k0, nk);
        }
        const int64_t len = std::min<int64_t>(every, nsteps - (int64_t)k * every);
        rc = chemo_step_n(s, len, stream);
    }
    if (nstore > 0) {
        s->kp.tape = KP::TapeOut{};
        eng_drop_graphs(s);
        if (rc == CHEMO_OK) rc = gather(s, all.pos + (size_t)nk * t->n * t->dim, nullptr, st);
    }
    return rc;
}

extern "C" int chemo_gradient(chemo_sim *s, const float *dL_dpos_final, const float *dL_dc_final, float *dL_dparams,
                              float *dL_dpos0, int mem_kind, void *stream)
{
    ChemoRange nvtx_range("chemo_gradient");
    if (!s) return eng_fail(CHEMO_EINVAL, "sim is NULL");
    chemo_tape *t = s->tape;
    if (!t) return eng_fail(CHEMO_EINVAL, "chemo_gradient: no recorded run (call chemo_record first)");
    if (mem_kind != CHEMO_MEM_HOST && mem_kind != CHEMO_MEM_DEVICE) return eng_fail(CHEMO_EINVAL, "bad mem_kind");
    if (!dL_dpos_final || !dL_dparams) return eng_fail(CHEMO_EINVAL, "dL_dpos_final and dL_dparams are required");
    cudaStream_t st = (cudaStream_t)stream;
    const int dim = t->dim;
    const int64_t n = t->n, G = t->G;
    const size_t pb = (size_t)std::max<int64_t>(n, 1) * dim * sizeof(float);
    const size_t gb = (size_t)std::max<int64_t>(G, 1) * sizeof(float);
    void *p;
    int r;
    bool rerun_any = false;
    for (const SegBuf &B : t->stored) rerun_any = rerun_any || !B.pos;
    if (rerun_any && !t->sb[0].pos) {
        // one block for both buffers, so that one tape (slot = step mod
        // 2 every) serves every re-run and its graphs are captured once
        const size_t E = (size_t)t->every, n1 = (size_t)std::max<int64_t>(n, 1), g1 = (size_t)std::max<int64_t>(G, 1);
        if ((r = alloc_steps(t, t->sb_all, 2 * E + 1))) return r;
        for (int b = 0; b < 2; ++b) {
            SegBuf &B = t->sb[b];
            const SegBuf &A = t->sb_all;
            B.pos = A.pos + (size_t)b * (E + 1) * n1 * dim;
            B.c = A.c + (size_t)b * E * g1;
            B.S = A.S + (size_t)b * E * n1;
            B.cnt = A.cnt + (size_t)b * E * t->cwords;
            B.gst = A.gst + (size_t)b * E * t->gwords;
            B.F = A.F + (size_t)b * E * n1 * dim;
        }
    }
    if (!t->s_fwd) {
        ATRY(cudaStreamCreateWithFlags(&t->s_fwd, cudaStreamNonBlocking));
        ATRY(cudaStreamCreateWithFlags(&t->s_rev, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            ATRY(cudaEventCreateWithFlags(&t->ev_ready[b], cudaEventDisableTiming));
            ATRY(cudaEventCreateWithFlags(&t->ev_done[b], cudaEventDisableTiming));
        }
        ATRY(cudaEventCreateWithFlags(&t->ev_start, cudaEventDisableTiming));
        ATRY(cudaEventCreateWithFlags(&t->ev_fwd_end, cudaEventDisableTiming));
        ATRY(cudaEventCreateWithFlags(&t->ev_rev_end, cudaEventDisableTiming));
        ATRY(cudaStreamCreateWithFlags(&t->s_pair, cudaStreamNonBlocking));
        ATRY(cudaEventCreateWithFlags(&t->ev_cells, cudaEventDisableTiming));
        ATRY(cudaEventCreateWithFlags(&t->ev_pairs, cudaEventDisableTiming));
        for (int k = 0; k < 2; ++k) {
            if ((r = talloc(t, &p, pb))) return r;
            t->lamX[k] = (float *)p;
            if ((r = talloc(t, &p, gb))) return r;
            t->lamC[k] = (float *)p;
        }
        if ((r = talloc(t, &p, pb))) return r;
        t->lamY = (float *)p;
        if ((r = talloc(t, &p, gb))) return r;
        t->lamS = (float *)p;
        t->pstride = (int64_t)blocks(std::max<int64_t>(n, 1) * 8);  // k_adj_cells: up to 8 threads per cell
        if ((r = talloc(t, &p, sizeof(double) * (2 + MAXS) * (size_t)t->pstride))) return r;
        t->dpar = (double *)p;
        if ((r = talloc(t, &p, sizeof(float) * (2 + MAXS)))) return r;
        t->dpf = (float *)p;
    }
    const cudaMemcpyKind in_kind = mem_kind == CHEMO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    // two streams after the caller's: re-runs on s_fwd, reverse sweeps on s_rev
    cudaStream_t sf = t->s_fwd, sr = t->s_rev;
    ATRY(cudaEventRecord(t->ev_start, st));
    ATRY(cudaStreamWaitEvent(sf, t->ev_start, 0));
    ATRY(cudaStreamWaitEvent(sr, t->ev_start, 0));
    int lx = 0, lc = 0;
    if (n) ATRY(cudaMemcpyAsync(t->lamX[lx], dL_dpos_final, (size_t)n * dim * sizeof(float), in_kind, sr));
    if (G) {
        if (dL_dc_final) ATRY(cudaMemcpyAsync(t->lamC[lc], dL_dc_final, (size_t)G * sizeof(float), in_kind, sr));
        else ATRY(cudaMemsetAsync(t->lamC[lc], 0, gb, sr));
    }
    ATRY(cudaMemsetAsync(t->dpar, 0, sizeof(double) * (2 + MAXS) * (size_t)t->pstride, sr));
    // the pair force is linear in inter: dF/dinter = F / inter (the cell list
    // is not built for the cutoff when inter = 0, and dL/dinter is then 0)
    const float f_unit = s->prm.inter != 0.f ? 1.f / s->prm.inter : 0.f;
    const int64_t end_step = t->step0 + t->nsteps;  // the recorded run's final step index
    // restores segment seg's checkpoint and re-runs it on sf, storing its states in B
    // (the particle kernel writes the states into buffer seg mod 2 through
    // the periodic tape, so chemo_step_n replays its graphs for every re-run)
    auto rerun = [&](int seg, SegBuf &B) -> int {
        const int64_t n0 = (int64_t)seg * t->every;
        const int64_t len = std::min<int64_t>(t->every, t->nsteps - n0);
        int rr;
        if ((rr = eng_ingest(s, t->ck_pos[seg], t->species, nullptr, CHEMO_MEM_DEVICE, sf))) return rr;
        if (G) ATRY(cudaMemcpyAsync(cur_field(s), t->ck_c[seg], gb, cudaMemcpyDeviceToDevice, sf));
        if ((rr = chemo_set_step_index(s, t->step0 + n0, sf))) return rr;
        if ((rr = chemo_step_n(s, len, sf))) return rr;
        return gather(s, B.pos + (size_t)len * n * dim, nullptr, sf);
    };
    // the tape points into this recording while re-runs are enqueued: cleared
    // (and the graphs that hold it dropped) on every way out
    struct TapeGuard {
        chemo_sim *s;
        bool on;
        ~TapeGuard()
        {
            if (on) {
                s->kp.tape = KP::TapeOut{};
                eng_drop_graphs(s);
            }
        }
    } guard{s, false};
    if (rerun_any) {
        eng_drop_graphs(s);
        KP::TapeOut &tp = s->kp.tape;
        tp = KP::TapeOut{};
        tp.pos = t->sb_all.pos;
        tp.c = t->sb_all.c;
        tp.F = t->sb_all.F;
        tp.S = t->sb_all.S;
        tp.cnt = t->sb_all.cnt;
        tp.gst = t->sb_all.gst;
        tp.s0 = (unsigned long long)t->step0;
        tp.period = tp.nk = 2ull * (unsigned long long)t->every;
        tp.pos_gap = (unsigned long long)t->every;
        tp.cwords = (int64_t)t->cwords;
        tp.gwords = (int64_t)t->gwords;
        guard.on = true;
    }
    auto is_stored = [&](int seg) { return t->stored[(size_t)seg].pos != nullptr; };
    bool sb_used[2] = {false, false};  // a reverse sweep has read the buffer (wait for it before refilling)
    if (!is_stored(t->nseg - 1)) {
        if ((r = rerun(t->nseg - 1, t->sb[(t->nseg - 1) & 1]))) return r;
        ATRY(cudaEventRecord(t->ev_ready[(t->nseg - 1) & 1], sf));
    }
    bool pairs_pending = false;  // a pair term on s_pair that sr has not waited for
    for (int seg = t->nseg - 1; seg >= 0; --seg) {
        const int64_t n0 = (int64_t)seg * t->every;
        const int64_t len = std::min<int64_t>(t->every, t->nsteps - n0);
        const bool stored = is_stored(seg);
        const SegBuf &B = stored ? t->stored[(size_t)seg] : t->sb[seg & 1];
        if (seg >= 1 && !is_stored(seg - 1)) {
            // re-run the previous segment into its buffer once the reverse
            // sweep that last read that buffer is done
            const int ob = (seg - 1) & 1;
            if (sb_used[ob]) ATRY(cudaStreamWaitEvent(sf, t->ev_done[ob], 0));
            if ((r = rerun(seg - 1, t->sb[ob]))) return r;
            ATRY(cudaEventRecord(t->ev_ready[ob], sf));
        }
        if (!stored) ATRY(cudaStreamWaitEvent(sr, t->ev_ready[seg & 1], 0));
        // reverse sweep over the segment (stream sr)
        for (int64_t k = len - 1; k >= 0; --k) {
            const unsigned long long step = (unsigned long long)(t->step0 + n0 + k);
            const float *Xn = B.pos + (size_t)k * n * dim;
            const float *Xn1 = B.pos + (size_t)(k + 1) * n * dim;
            const float *cn = G ? B.c + (size_t)k * G : nullptr;
            KP kp = eng_view(s);  // constants only: the buffers come from B
            // 1. PDE transpose (substeps), lambda_S
            if (G && kp.pde_multi) {
                // 2D: the transpose of the mirror-ghost operator is tau L tau^-1, so
                // nu = lambda / tau runs the forward substeps (several per launch);
                // lambda_S / tau is the mean of the substeps' nu
                int left = kp.substeps;
                for (int l = 0; l < kp.pde_launches; ++l) {
                    const int nsub = (left + (kp.pde_launches - l) - 1) / (kp.pde_launches - l);
                    ATRY(launch_pde_multi(kp, t->lamC[lc], t->lamC[lc ^ 1], nsub, 0, t->lamS, l == 0,
                                          1.f / (float)kp.substeps, 1, sr));
                    left -= nsub;
                    lc ^= 1;
                }
            } else if (G) {
                const int ss = kp.substeps;
                for (int m = 0; m < ss; ++m) {
                    k_adj_pde<<<blocks(G), ATPB, 0, sr>>>(kp, t->lamC[lc], t->lamC[lc ^ 1], t->lamS, 1.f / ss, m == 0);
                    ATRY(cudaGetLastError());
                    lc ^= 1;
                }
            }
            // the cell list of X^n and its pair force, saved by the re-run
            kp.S = B.S + (size_t)k * n;
            kp.cnt_cur = B.cnt + (size_t)k * t->cwords;
            kp.gstart = B.gst + (size_t)k * t->gwords;
            const float *Fk = B.F + (size_t)k * n * dim;
            // 2-5. per-cell terms, then the pair term; the pair term only adds
            // to lambda_X^n and reads lambda_Y, so it runs on its own stream
            // beside the next (earlier) step's PDE transpose, and the next
            // per-cell kernel (which rewrites lambda_Y) waits for it
            if (n) {
                if (pairs_pending) {
                    ATRY(cudaStreamWaitEvent(sr, t->ev_pairs, 0));
                    pairs_pending = false;
                }
                if (dim == 2)
                    k_adj_cells<2><<<blocks(n * 4), ATPB, 0, sr>>>(kp, Xn, Xn1, t->species, cn, t->lamX[lx], t->lamS, Fk, f_unit,
                                                             t->lamY, t->lamX[lx ^ 1], t->lamC[lc], step, t->dpar,
                                                             t->pstride, G ? 1 : 0, kp.pde_multi, t->layer_id);
                else
                    k_adj_cells<3><<<blocks(n * 8), ATPB, 0, sr>>>(kp, Xn, Xn1, t->species, cn, t->lamX[lx], t->lamS, Fk, f_unit,
                                                             t->lamY, t->lamX[lx ^ 1], t->lamC[lc], step, t->dpar,
                                                             t->pstride, G ? 1 : 0, kp.pde_multi, t->layer_id);
                ATRY(cudaGetLastError());
                if (kp.pairs) {
                    cudaStream_t sp2 = t->s_pair;
                    ATRY(cudaEventRecord(t->ev_cells, sr));
                    ATRY(cudaStreamWaitEvent(sp2, t->ev_cells, 0));
                    // walls: the half window (each pair once; the 3^d bins of
                    // a search mode other than 2 are needed for it)
                    const bool half = !kp.periodic && kp.search != 2;
                    const unsigned nbk = blocks(n * APC);
                    if (dim == 2) {
                        if (kp.periodic) k_adj_pairs<2, true, false><<<nbk, ATPB, 0, sp2>>>(kp, t->lamY, t->lamX[lx ^ 1]);
                        else if (half) k_adj_pairs<2, false, true><<<nbk, ATPB, 0, sp2>>>(kp, t->lamY, t->lamX[lx ^ 1]);
                        else k_adj_pairs<2, false, false><<<nbk, ATPB, 0, sp2>>>(kp, t->lamY, t->lamX[lx ^ 1]);
                    } else {
                        if (kp.periodic) k_adj_pairs<3, true, false><<<nbk, ATPB, 0, sp2>>>(kp, t->lamY, t->lamX[lx ^ 1]);
                        else if (half) k_adj_pairs<3, false, true><<<nbk, ATPB, 0, sp2>>>(kp, t->lamY, t->lamX[lx ^ 1]);
                        else k_adj_pairs<3, false, false><<<nbk, ATPB, 0, sp2>>>(kp, t->lamY, t->lamX[lx ^ 1]);
                    }
                    ATRY(cudaGetLastError());
                    ATRY(cudaEventRecord(t->ev_pairs, sp2));
                    pairs_pending = true;
                }
            }
            lx ^= 1;
        }
        if (pairs_pending) {  // the segment's buffer is free once its last pair term is done
            ATRY(cudaStreamWaitEvent(sr, t->ev_pairs, 0));
            pairs_pending = false;
        }
        if (!stored) {
            ATRY(cudaEventRecord(t->ev_done[seg & 1], sr));
            sb_used[seg & 1] = true;
        }
    }
    if (guard.on) {  // every re-run is enqueued
        s->kp.tape = KP::TapeOut{};
        eng_drop_graphs(s);
        guard.on = false;
    }
    // join both streams back into the caller's
    ATRY(cudaEventRecord(t->ev_fwd_end, sf));
    ATRY(cudaEventRecord(t->ev_rev_end, sr));
    ATRY(cudaStreamWaitEvent(st, t->ev_fwd_end, 0));
    ATRY(cudaStreamWaitEvent(st, t->ev_rev_end, 0));
    // outputs
    const int np = 2 + t->ns;
    float *dpf = t->dpf;
    k_params_out<<<1, 32 * (2 + MAXS), 0, st>>>(t->dpar, t->pstride, dpf, np);
    ATRY(cudaGetLastError());
    const cudaMemcpyKind out_kind = mem_kind == CHEMO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    ATRY(cudaMemcpyAsync(dL_dparams, dpf, sizeof(float) * np, out_kind, st));
    if (dL_dpos0 && n) ATRY(cudaMemcpyAsync(dL_dpos0, t->lamX[lx], (size_t)n * dim * sizeof(float), out_kind, st));
    // leave the simulation at the final state of the recorded run
    if ((r = eng_ingest(s, t->ck_pos[t->nseg], t->species, nullptr, CHEMO_MEM_DEVICE, st))) return r;
    if (G) ATRY(cudaMemcpyAsync(cur_field(s), t->ck_c[t->nseg], gb, cudaMemcpyDeviceToDevice, st));
    if ((r = chemo_set_step_index(s, end_step, stream))) return r;
    if (mem_kind == CHEMO_MEM_HOST) ATRY(cudaStreamSynchronize(st));
    return CHEMO_OK;
}
