// chemo_engine.h -- the simulation object shared by the engine translation
// units (chemo_capi.cu: forward; adjoint.cu: recording and adjoint). Not part
// of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "../../include/chemo.h"
#include "chemo_internal.cuh"

using chemo::KP;

struct chemo_tape;  // recorded run (adjoint.cu)

// Named range of a library call for timeline profilers (NVTX; a no-op unless
// a profiler is attached).
struct ChemoRange {
    explicit ChemoRange(const char *name) { nvtxRangePushA(name); }
    ~ChemoRange() { nvtxRangePop(); }
    ChemoRange(const ChemoRange &) = delete;
    ChemoRange &operator=(const ChemoRange &) = delete;
};

// Source of device buffers: the allocator given to chemo_set_allocator, or
// cudaMalloc / cudaFree when both callbacks are NULL.
struct DevMem {
    chemo_alloc_fn alloc = nullptr;
    chemo_release_fn release = nullptr;
    void *ctx = nullptr;
};

// A device buffer with the size it was allocated with.
struct DevBuf {
    void *ptr;
    size_t bytes;
};

struct chemo_sim {
    chemo_params prm{};
    KP kp{};
    uint32_t *cnt8[2] = {nullptr, nullptr};  // packed bin counts, double buffered
    int cntp = 0;                // cnt8[cntp] describes the sorted state
    int cur = 0;                 // c[cur] holds c^n
    int64_t step = 0;            // host mirror of the next step index
    int launches_per_step = 0;
    cudaStream_t aux = nullptr;  // second stream for the PDE (lowest priority)
    cudaStream_t hp = nullptr;   // the particle kernels beside it (highest priority)
    cudaEvent_t ev_hp = nullptr;
    cudaStream_t cap = nullptr;  // capture stream for graphs
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t graph[2][2][2] = {};  // [2-step, 16-step][grid parity][count parity]
    DevMem mem;                  // the allocator in force at creation
    std::vector<DevBuf> allocs;
    int64_t bytes = 0;
    void *scratch = nullptr;     // staging for host transfers and stage outputs
    size_t scratch_bytes = 0;
    chemo_tape *tape = nullptr;  // recorded run for the adjoint (adjoint.cu)
    std::vector<int64_t> layer_off_host;  // replicate offsets (layers + 1), host copy
    int64_t capacity = 0;        // cells the buffers hold (kp.n <= capacity; kp.n changes only in sub-domains)
};

// Engine services used by adjoint.cu (implemented in chemo_capi.cu).
int eng_fail(int status, const char *fmt, ...);
// The process-wide allocator setting now.
DevMem eng_allocator();
// bytes (rounded up to 256) of device memory from m; CHEMO_OK or CHEMO_ENOMEM
// with the last error set. *p is NULL on failure; *rounded gets the size
// release must be given.
int eng_mem_alloc(const DevMem &m, void **p, size_t bytes, size_t *rounded);
// Gives back a buffer of eng_mem_alloc (p may be NULL).
void eng_mem_release(const DevMem &m, void *p, size_t bytes);
int eng_dalloc(chemo_sim *s, void **p, size_t bytes);
// Device scratch of at least `bytes` owned by the simulation (reused by every call).
int eng_scratch(chemo_sim *s, size_t bytes, void **p);
KP eng_view(const chemo_sim *s);
int eng_enqueue_step(chemo_sim *s, cudaStream_t st, int *launches);
int eng_ingest(chemo_sim *s, const float *pos, const uint8_t *sp, const float *disp, int mem_kind, cudaStream_t st);
void eng_drop_graphs(chemo_sim *s);
// Model constants of params into kp (species tables, noise, ...).
void eng_fill_model(const chemo_params &p, KP &kp);
// Releases a recorded run (adjoint.cu).
void chemo_tape_free(chemo_tape *t);
