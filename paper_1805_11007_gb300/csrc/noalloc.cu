// noalloc.cu -- pair forces of a caller's particle set with no device
// allocation: the cell list lives in one fixed-size array in device global
// memory that is part of the loaded library.
//
// Who needs this: code that must not call cudaMalloc at the point where it
// wants forces -- for example a host application that hands this library a
// fixed memory budget and forbids new device allocations after start-up, a
// real-time loop where an allocation (which may synchronise the device) would
// break its timing, or a plug-in running inside another framework's
// allocator. Such a caller passes device buffers for the inputs and the
// output; everything else the computation needs comes from g_scratch below.
//
// Costs of the design: every GPU that loads the library holds the array
// (NOALLOC_BYTES) until the process exits, the array is shared by all calls
// (calls whose kernels overlap on the GPU race on it: keep them on one stream
// or otherwise ordered), and the problem size is capped (NOALLOC_MAX_N
// particles, NOALLOC_MAX_BINS cell-list bins). The particle cap keeps every
// 16-bit bin count below its wrap-around, even with all particles in one bin.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/chemo.h"
#include "chemo_internal.cuh"

using namespace chemo;

namespace {

// A bin holds at most BIN_COUNT_MAX particles (16-bit packed counts), so at
// most that many particles are accepted: one bin can then never overflow.
constexpr int64_t NOALLOC_MAX_N = BIN_COUNT_MAX;
static_assert(NOALLOC_MAX_N <= (int64_t)BIN_COUNT_MAX, "a single bin could overflow its 16-bit count");
constexpr int64_t NOALLOC_CAP = NOALLOC_MAX_N + 1;  // particle slots (a multiple of 16)
constexpr int64_t NOALLOC_MAX_BINS = (int64_t)1 << 18;  // a multiple of 8
constexpr int64_t NOALLOC_MAX_GROUPS = NOALLOC_MAX_BINS / 8;
constexpr int64_t NOALLOC_MAX_TILES = (NOALLOC_MAX_GROUPS + 2047) / 2048;

// Sub-array sizes in bytes, each a multiple of 256.
constexpr size_t SZ_STATE = (size_t)NOALLOC_CAP * sizeof(float4);            // S and U
constexpr size_t SZ_SLOT = (size_t)NOALLOC_CAP * sizeof(uint32_t);
constexpr size_t SZ_CNT = (size_t)NOALLOC_MAX_BINS / 2 * sizeof(uint32_t);      // 16-bit counts
constexpr size_t SZ_GSTART = ((size_t)NOALLOC_MAX_GROUPS + 256) * sizeof(uint32_t);
constexpr size_t SZ_TILES = 256 * ((NOALLOC_MAX_TILES * 8 + 255) / 256);
constexpr size_t SZ_CTL = 256;
constexpr size_t NOALLOC_BYTES = 2 * SZ_STATE + SZ_SLOT + 2 * SZ_CNT + SZ_GSTART + SZ_TILES + SZ_CTL;

static_assert(SZ_TILES >= NOALLOC_MAX_TILES * sizeof(unsigned long long), "tile table too small");
static_assert(SZ_STATE % 256 == 0 && SZ_SLOT % 256 == 0 && SZ_CNT % 256 == 0 && SZ_GSTART % 256 == 0,
              "sub-arrays must keep 256-byte alignment");

}  // namespace

// The scratch array (about 3.4 MB). Host code must not use its name as an
// address: it is a host-side stand-in. The device address is obtained once
// per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[NOALLOC_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

// Device address of g_scratch on the current device (looked up on first use
// per device, with that device current).
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return chemo_internal_fail(CHEMO_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return chemo_internal_fail(CHEMO_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return chemo_internal_fail(CHEMO_ECUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                     : "cudaGetSymbolAddress returned NULL");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return CHEMO_OK;
}

}  // namespace

extern "C" int chemo_forces_noalloc(const chemo_params *params, int64_t n, const float *pos, const uint8_t *species,
                                    float *F_out, void *stream)
{
    KP kp{};
    if (int r = chemo_internal_build_kp(params, n, &kp)) return r;
    if (n > NOALLOC_MAX_N)
        return chemo_internal_fail(CHEMO_EINVAL, "chemo_forces_noalloc: n exceeds the limit of 65535 particles");
    if (kp.bin_slots > NOALLOC_MAX_BINS)
        return chemo_internal_fail(CHEMO_EINVAL, "chemo_forces_noalloc: the cell list needs more than 262144 bins "
                                                 "(box too large for the cutoff); use chemo_create instead");
    if (n == 0) return CHEMO_OK;
    if (!pos || !species || !F_out) return chemo_internal_fail(CHEMO_EINVAL, "pos, species and F_out are required");
    // the half window needs a buffer of force sums: the full 3^d window per
    // lane gives the same forces bit for bit
    if (kp.search == 4) kp.search = 3;
    kp.Fh = nullptr;
    void *base = nullptr;
    if (int r = scratch_address(&base)) return r;
    unsigned char *b = static_cast<unsigned char *>(base);
    kp.S = reinterpret_cast<float4 *>(b);
    kp.U = reinterpret_cast<float4 *>(b + SZ_STATE);
    kp.slot = reinterpret_cast<uint32_t *>(b + 2 * SZ_STATE);
    uint32_t *cnt0 = reinterpret_cast<uint32_t *>(b + 2 * SZ_STATE + SZ_SLOT);
    uint32_t *cnt1 = reinterpret_cast<uint32_t *>(b + 2 * SZ_STATE + SZ_SLOT + SZ_CNT);
    kp.gstart = reinterpret_cast<uint32_t *>(b + 2 * SZ_STATE + SZ_SLOT + 2 * SZ_CNT);
    kp.tiles = reinterpret_cast<unsigned long long *>(b + 2 * SZ_STATE + SZ_SLOT + 2 * SZ_CNT + SZ_GSTART);
    uint32_t *ctl = reinterpret_cast<uint32_t *>(b + 2 * SZ_STATE + SZ_SLOT + 2 * SZ_CNT + SZ_GSTART + SZ_TILES);
    kp.tile_ctr = ctl;
    kp.scan_seq = ctl + 1;
    kp.err = ctl + 2;
    kp.step = reinterpret_cast<unsigned long long *>(ctl + 4);
    kp.dS = kp.dU = nullptr;
    kp.c[0] = kp.c[1] = nullptr;
    kp.srcg = kp.Rg = nullptr;
    kp.has_grid = 0;  // forces only: no deposit in the scatter
    cudaStream_t st = (cudaStream_t)stream;
    // The array keeps the previous call's contents: clear the counts that the
    // binning adds to, the scan's tile table and its control words.
    const size_t cbytes = (size_t)kp.bin_slots / 2 * sizeof(uint32_t);
    cudaError_t e = cudaMemsetAsync(cnt1, 0, cbytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(kp.tiles, 0, SZ_TILES, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, SZ_CTL, st);
    // bin the particles: count into cnt1, scan (clears cnt0), place into S
    kp.cnt_cur = cnt0;
    kp.cnt_nxt = cnt1;
    if (e == cudaSuccess) e = launch_pack(kp, pos, species, nullptr, st, nullptr);
    if (e == cudaSuccess) e = launch_scan(kp, st, nullptr);
    if (e == cudaSuccess) e = launch_scatter(kp, 0, 0, st, nullptr);
    // pair force over the binned state (cnt1 now describes S)
    kp.cnt_cur = cnt1;
    kp.cnt_nxt = cnt0;
    if (e == cudaSuccess) e = launch_stage_forces(kp, F_out, nullptr, nullptr, st);
    if (e != cudaSuccess) return chemo_internal_fail(CHEMO_ECUDA, cudaGetErrorString(e));
    return CHEMO_OK;
}
