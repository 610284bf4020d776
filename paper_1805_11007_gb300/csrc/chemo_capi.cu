// chemo_capi.cu -- engine and C ABI (include/chemo.h) of the GB300
// chemotaxis step (arXiv:1805.11007): parameter validation, cell-list and
// grid layout, device buffers, the per-step launch sequence (PDE overlapped
// with the particle kernel on a second stream when one substep suffices) and
// CUDA-graph replay of repeated steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/chemo.h"
#include "chemo_engine.h"
#include "chemo_internal.cuh"

using namespace chemo;

namespace {

thread_local char g_last_error[512] = "";

int fail(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return status;
}

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? CHEMO_ENOMEM : CHEMO_ECUDA,    \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

__global__ void k_set_u64(unsigned long long *p, unsigned long long v) { *p = v; }

}  // namespace


namespace {

std::mutex g_alloc_mu;
DevMem g_alloc;  // the setting of chemo_set_allocator, guarded by g_alloc_mu

int dalloc(chemo_sim *s, void **p, size_t bytes)
{
    size_t b = 0;
    if (int r = eng_mem_alloc(s->mem, p, bytes, &b)) return r;
    s->allocs.push_back({*p, b});
    s->bytes += (int64_t)b;
    return CHEMO_OK;
}

int scratch(chemo_sim *s, size_t bytes, void **out)
{
    if (bytes > s->scratch_bytes) {
        if (s->scratch) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return fail(CHEMO_ECUDA, "sync: %s", cudaGetErrorString(e));
            eng_mem_release(s->mem, s->scratch, s->scratch_bytes);
            s->bytes -= (int64_t)s->scratch_bytes;
            s->scratch = nullptr;
            s->scratch_bytes = 0;
        }
        size_t b = 0;
        if (int r = eng_mem_alloc(s->mem, &s->scratch, bytes, &b)) return r;
        s->scratch_bytes = b;
        s->bytes += (int64_t)b;
    }
    *out = s->scratch;
    return CHEMO_OK;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double grid_h(const chemo_params &p, int a)
{
    const double L = p.hi[a] - p.lo[a];
    return p.pde_bc == 2 ? L / p.grid[a] : L / (p.grid[a] - 1);
}

int resolve_substeps(const chemo_params &p)
{
    if (p.pde_substeps > 0) return p.pde_substeps;
    double lam = 0.0;
    for (int a = 0; a < p.dim; ++a) {
        const double h = grid_h(p, a);
        lam += 2.0 * (double)p.Dc * p.dt / (h * h);
    }
    const int s = (int)std::ceil(lam / 0.9);
    return s < 1 ? 1 : s;
}

// Validates p; on success fills the model constants of kp (not the layout).
int check_params(const chemo_params &p)
{
    if (p.struct_size != sizeof(chemo_params))
        return fail(CHEMO_EINVAL, "chemo_params.struct_size = %u, expected %zu", p.struct_size, sizeof(chemo_params));
    if (p.dim != 2 && p.dim != 3) return fail(CHEMO_EINVAL, "dim must be 2 or 3 (got %d)", p.dim);
    if (p.boundary != 0 && p.boundary != 1) return fail(CHEMO_EINVAL, "boundary must be 0 or 1");
    if (p.n_species < 1 || p.n_species > CHEMO_MAX_SPECIES) return fail(CHEMO_EINVAL, "n_species must be 1..8");
    for (int a = 0; a < p.dim; ++a)
        if (!(p.hi[a] > p.lo[a]) || !std::isfinite(p.lo[a]) || !std::isfinite(p.hi[a]))
            return fail(CHEMO_EINVAL, "empty or non-finite box on axis %d", a);
    if (!(p.dt > 0.0) || !std::isfinite(p.dt)) return fail(CHEMO_EINVAL, "dt must be positive");
    for (int s = 0; s < p.n_species; ++s) {
        if (!(p.diameter[s] >= 0.f) || !(p.D[s] >= 0.f)) return fail(CHEMO_EINVAL, "species %d: negative diameter or D", s);
        if (p.react_to[s] < 0 || p.react_to[s] >= p.n_species) return fail(CHEMO_EINVAL, "species %d: react_to out of range", s);
    }
    if (p.cutoff_mode != 0 && p.cutoff_mode != 1) return fail(CHEMO_EINVAL, "cutoff_mode must be 0 or 1");
    if (!(p.cutoff_factor >= 0.f)) return fail(CHEMO_EINVAL, "cutoff_factor must be >= 0");
    if (p.chem_mode != 0 && p.chem_mode != 1) return fail(CHEMO_EINVAL, "chem_mode must be 0 or 1");
    if (p.search_mode < 0 || p.search_mode > 4) return fail(CHEMO_EINVAL, "search_mode must be 0, 1, 2, 3 or 4");
    if (p.warp_runs < 0 || p.warp_runs > 32) return fail(CHEMO_EINVAL, "warp_runs must be 0..32");
    if (p.block_threads != 0 && p.block_threads != 128 && p.block_threads != 256 && p.block_threads != 512)
        return fail(CHEMO_EINVAL, "block_threads must be 0, 128, 256 or 512");
    if (p.move_scheme != 0 && p.move_scheme != 1) return fail(CHEMO_EINVAL, "move_scheme must be 0 or 1");
    if (p.hard_sphere != 0 && p.hard_sphere != 1) return fail(CHEMO_EINVAL, "hard_sphere must be 0 or 1");
    if (p.deposit_kernel != 0 && p.deposit_kernel != 1) return fail(CHEMO_EINVAL, "deposit_kernel must be 0 or 1");
    if (!(p.kde_range >= 0.f) || !std::isfinite(p.kde_range)) return fail(CHEMO_EINVAL, "kde_range must be >= 0");
    if (p.deposit_kernel == 1) {
        if (p.chem_mode != 0) return fail(CHEMO_EINVAL, "deposit_kernel 1 needs the grid (chem_mode 0)");
        for (int s = 0; s < p.n_species; ++s)
            if ((p.secrete[s] != 0.f || p.consume[s] != 0.f) && !(p.diameter[s] > 0.f))
                return fail(CHEMO_EINVAL, "deposit_kernel 1: species %d deposits but has no diameter (bandwidth)", s);
    }
    if (p.bin_order < 0 || p.bin_order > 2) return fail(CHEMO_EINVAL, "bin_order must be 0, 1 or 2");
    if (p.pde_overlap < 0 || p.pde_overlap > 2) return fail(CHEMO_EINVAL, "pde_overlap must be 0, 1 or 2");
    if (p.chem_mode == 0) {
        if (p.pde_bc < 0 || p.pde_bc > 2) return fail(CHEMO_EINVAL, "pde_bc must be 0, 1 or 2");
        if ((p.pde_bc == 2) != (p.boundary == 1))
            return fail(CHEMO_EINVAL, "pde_bc = 2 (periodic) goes with boundary = 1 and only with it");
        for (int a = 0; a < p.dim; ++a)
            if (p.grid[a] < 3) return fail(CHEMO_EINVAL, "grid[%d] = %d: need at least 3 nodes", a, p.grid[a]);
        if (p.pde_substeps < 0) return fail(CHEMO_EINVAL, "pde_substeps must be >= 0");
    }
    return CHEMO_OK;
}

double max_cutoff(const chemo_params &p)
{
    double m = 0.0;
    for (int s = 0; s < p.n_species; ++s)
        for (int t = 0; t < p.n_species; ++t)
            m = std::max(m, (double)p.cutoff_factor * 0.5 * ((double)p.diameter[s] + (double)p.diameter[t]));
    return m;
}

// Model constants that chemo_set_params may change.
void fill_model(const chemo_params &p, KP &kp)
{
    kp.ns = p.n_species;
    const double hd = [&] {
        double v = 1.0;
        if (p.chem_mode == 0)
            for (int a = 0; a < p.dim; ++a) v *= grid_h(p, a);
        return v;
    }();
    for (int s = 0; s < MAXS; ++s) {
        for (int t = 0; t < MAXS; ++t) {
            const int i = s * MAXS + t;
            kp.rc2[i] = 0.f;
            kp.inv_eps[i] = 0.f;
            kp.amp_f[i] = 0.f;
            kp.shift[i] = 0.f;
            if (s < p.n_species && t < p.n_species) {
                const double eps = 0.5 * ((double)p.diameter[s] + (double)p.diameter[t]);
                if (eps > 0.0) {
                    const double rc = (double)p.cutoff_factor * eps;
                    kp.rc2[i] = (float)(rc * rc);
                    kp.inv_eps[i] = (float)(1.0 / eps);
                    kp.amp_f[i] = (float)((double)p.inter / eps);
                    kp.shift[i] = p.cutoff_mode == 1 ? (float)std::exp(-(double)p.cutoff_factor) : 0.f;
                }
            }
        }
        const bool in = s < p.n_species;
        kp.noise[s] = in ? (float)std::sqrt(2.0 * (double)p.D[s] * p.dt) : 0.f;
        kp.chem[s] = in ? p.chi * p.chemotactic[s] : 0.f;
        kp.chemotactic_f[s] = in ? p.chemotactic[s] : 0.f;
        kp.src[s] = in ? (float)((double)p.secrete[s] * p.dt / hd) : 0.f;
        kp.cons[s] = in ? (float)((double)p.consume[s] / hd) : 0.f;
        kp.rk0[s] = in ? p.react_k0[s] : 0.f;
        kp.rkc[s] = in ? p.react_kc[s] : 0.f;
        kp.rto[s] = in ? p.react_to[s] : s;
    }
    // search radius per species: its largest cutoff against any species, with
    // a 1e-3 relative margin over FP32 rounding of the bin-relative position
    for (int s = 0; s < MAXS; ++s) {
        double m = 0.0;
        if (s < p.n_species)
            for (int t = 0; t < p.n_species; ++t)
                m = std::max(m, (double)p.cutoff_factor * 0.5 * ((double)p.diameter[s] + (double)p.diameter[t]));
        const double r = m * (1.0 + 1e-3);
        kp.rsp2[s] = (float)(r * r);
    }
    // fixed-point quantum of the pair-force sum: 2^-25 of the largest pair
    // force magnitude inter/eps (terms never exceed it, so 16 of them fit an
    // int32)
    double fmax = 0.0;
    for (int i = 0; i < MAXS * MAXS; ++i) fmax = std::max(fmax, (double)std::fabs(kp.amp_f[i]));
    if (!(fmax > 0.0)) fmax = 1.0;
    kp.fq = (float)std::ldexp(fmax, -25);
    kp.fq_inv = (float)(1.0 / (double)kp.fq);
    kp.inter_f = p.inter;
    kp.reactions = p.reactions ? 1 : 0;
    // variants: tamed move, hard-sphere tables, kernel density constants
    kp.move_scheme = p.move_scheme;
    kp.hard_sphere = p.hard_sphere;
    for (int s = 0; s < MAXS; ++s)
        for (int t = 0; t < MAXS; ++t) {
            const int i = s * MAXS + t;
            const bool in = s < p.n_species && t < p.n_species;
            kp.hs_contact[i] = in ? (float)(0.5 * ((double)p.diameter[s] + (double)p.diameter[t])) : 0.f;
            const double Ds = in ? (double)p.D[s] : 0.0, Dt = in ? (double)p.D[t] : 0.0;
            kp.hs_share[i] = (float)(Ds + Dt > 0.0 ? Ds / (Ds + Dt) : 0.5);
        }
    kp.kde = p.deposit_kernel == 1 ? 1 : 0;
    const double krange = p.kde_range > 0.f ? (double)p.kde_range : 3.0;
    for (int s = 0; s < MAXS; ++s) {
        const double sig = s < p.n_species ? (double)p.diameter[s] : 0.0;
        const bool dep = s < p.n_species && (p.secrete[s] != 0.f || p.consume[s] != 0.f) && sig > 0.0;
        const double norm = dep ? std::pow(2.0 * 3.14159265358979323846 * sig * sig, -0.5 * p.dim) : 0.0;
        kp.kde_r2[s] = dep ? (float)(krange * sig * krange * sig) : -1.f;
        kp.kde_c[s] = dep ? (float)(0.5 / (sig * sig)) : 0.f;
        kp.kde_src[s] = dep ? (float)(p.dt * (double)p.secrete[s] * norm) : 0.f;
        kp.kde_cons[s] = dep ? (float)((double)p.consume[s] * norm) : 0.f;
    }
    double smax = 0.0, rmax = 0.0;
    for (int s = 0; s < MAXS; ++s) {
        smax = std::max(smax, (double)std::fabs(kp.kde_src[s]));
        rmax = std::max(rmax, (double)std::fabs(kp.kde_cons[s]));
    }
    kp.kde_qs = (float)std::ldexp(smax > 0.0 ? smax : 1.0, -24);
    kp.kde_qr = (float)std::ldexp(rmax > 0.0 ? rmax : 1.0, -24);
    double kr = 0.0;
    for (int s = 0; s < MAXS; ++s) kr = std::max(kr, kp.kde_r2[s] > 0.f ? std::sqrt((double)kp.kde_r2[s]) : 0.0);
    kp.kde_rmax = (float)(kr * (1.0 + 1e-4));  // margin over the rounding of bin edges
    kp.kde_qs_inv = (float)(1.0 / (double)kp.kde_qs);
    kp.kde_qr_inv = (float)(1.0 / (double)kp.kde_qr);
    kp.dt = (float)p.dt;
    kp.dt_d = p.dt;
    kp.seed_lo = (uint32_t)p.seed;
    kp.seed_hi = (uint32_t)(p.seed >> 32);
    kp.chem_mode = p.chem_mode;
    for (int a = 0; a < 3; ++a) kp.fixed_g[a] = a < p.dim ? p.fixed_grad[a] : 0.f;
    kp.Dc = p.Dc;
    kp.gamma = p.gamma;
}

// Cell-list layout: bin side >= r_c (3^d search) or >= 2 r_c (2^d search),
// row-major or Z-order storage.
int fill_layout(const chemo_params &p, int64_t n, KP &kp)
{
    kp.dim = p.dim;
    kp.scan_spins = 1u << 22;  // look-back polls (~0.1 s) before the scan gives up
    kp.periodic = p.boundary == 1;
    for (int a = 0; a < 3; ++a) {
        kp.lo[a] = a < p.dim ? (float)p.lo[a] : 0.f;
        kp.hi[a] = a < p.dim ? (float)p.hi[a] : 0.f;
        kp.L[a] = a < p.dim ? (float)(p.hi[a] - p.lo[a]) : 0.f;
        kp.halfL[a] = 0.5f * kp.L[a];
        kp.nb[a] = 1;
        kp.inv_b[a] = 0.f;
        kp.bside[a] = 0.f;
    }
    const double rc_force = max_cutoff(p);
    const bool pairs = rc_force > 0.0 && p.inter != 0.f;
    double contact = 0.0;  // hard-sphere contact distance: searched like a cutoff
    if (p.hard_sphere)
        for (int s = 0; s < p.n_species; ++s)
            for (int t = 0; t < p.n_species; ++t)
                contact = std::max(contact, 0.5 * ((double)p.diameter[s] + (double)p.diameter[t]));
    const double rc = std::max(pairs ? rc_force : 0.0, contact);
    const bool search_on = rc > 0.0;
    // automatic: the upper half of the 3^d window searched per lane, each pair
    // once (fastest on the clump, walls and ensemble workloads; the warp search
    // wins only in the densest states and is left to the autotuner)
    int search = !pairs ? 1 : (p.search_mode == 0 ? 4 : p.search_mode);
    kp.pairs = pairs ? 1 : 0;
    double bmin;
    if (search_on) {
        bmin = (search == 2 ? 2.0 : 1.0) * rc * (1.0 + 1.0 / 4096.0);
        if (p.bin_side > 0.f) {
            if ((double)p.bin_side < bmin)
                return fail(CHEMO_EINVAL, "bin_side %g is below the %s search minimum %g", (double)p.bin_side,
                            search == 2 ? "2^d" : "3^d", bmin);
            bmin = p.bin_side;
        }
    } else {
        // no interaction: bins only order the particles (about 2^d per bin)
        double vol = 1.0;
        for (int a = 0; a < p.dim; ++a) vol *= p.hi[a] - p.lo[a];
        const double per_layer = (double)std::max<int64_t>(n, 1) / (double)std::max(kp.layers, 1);
        bmin = p.bin_side > 0.f ? (double)p.bin_side
                                : std::pow(vol * (double)(1 << p.dim) / std::max(per_layer, 1.0), 1.0 / p.dim);
    }
    double kde_radius = 0.0;  // largest truncation radius of the density kernel
    if (p.deposit_kernel == 1) {  // the density window spans at most 3 bins per side
        const double krange = p.kde_range > 0.f ? (double)p.kde_range : 3.0;
        for (int s = 0; s < p.n_species; ++s) kde_radius = std::max(kde_radius, krange * (double)p.diameter[s]);
        bmin = std::max(bmin, kde_radius / 3.0);
    }
    int64_t total = 1;
    for (int a = 0; a < p.dim; ++a) {
        const double L = p.hi[a] - p.lo[a];
        double m = std::floor(L / bmin);
        if (m < 1.0) m = 1.0;
        if (!search_on) m = std::min(m, 1024.0);
        if (m > 65535.0) return fail(CHEMO_EINVAL, "axis %d needs %g bins: cutoff too small for the box", a, m);
        kp.nb[a] = (int)m;
        kp.inv_b[a] = (float)((double)kp.nb[a] / L);
        kp.bside[a] = (float)(L / kp.nb[a]);
        total *= kp.nb[a];
    }
    if (p.dim == 2) kp.nb[2] = std::max(kp.layers, 1);  // replicates as the third bin index
    kp.kde_win = 0;
    if (p.deposit_kernel == 1) {
        for (int a = 0; a < p.dim; ++a)
            kp.kde_win = std::max(kp.kde_win, (int)std::ceil(kde_radius / (double)kp.bside[a] * (1.0 - 1e-9)));
        if (kp.periodic)
            for (int a = 0; a < p.dim; ++a)
                if (kp.nb[a] < 2 * kp.kde_win + 1)
                    return fail(CHEMO_EINVAL, "periodic axis %d holds %d bins: too few for the density kernel's range",
                                a, kp.nb[a]);
    }
    if (search_on && kp.periodic) {
        for (int a = 0; a < p.dim; ++a) {
            if (search != 2 && kp.nb[a] < 3)
                return fail(CHEMO_EINVAL, "periodic axis %d holds %d bins of side >= r_c; need >= 3 (box too small "
                                          "for the cutoff; try search_mode 2)", a, kp.nb[a]);
            if (search == 2 && kp.nb[a] < 3)
                return fail(CHEMO_EINVAL, "periodic axis %d holds %d bins of side >= 2 r_c; need >= 3", a, kp.nb[a]);
        }
    }
    if (p.bin_order == 2) return fail(CHEMO_ENOTSUP, "Z-order bin storage is not supported; bins are row-major");
    // row-major bins, rows padded to a multiple of 8 so that a group of 8
    // bins never straddles two rows
    kp.px = (kp.nb[0] + 7) & ~7;
    const int64_t slots = (int64_t)kp.px * kp.nb[1] * kp.nb[2];
    if (slots > ((int64_t)1 << 31)) return fail(CHEMO_EINVAL, "cell list would need %lld bins", (long long)slots);
    kp.bin_slots = slots;
    kp.ngroups = slots / 8;
    kp.search = search;
    kp.warp_runs = p.warp_runs > 0 ? p.warp_runs : 12;
    kp.bt = p.block_threads > 0 ? p.block_threads : 256;
    return CHEMO_OK;
}

int fill_grid(const chemo_params &p, KP &kp)
{
    kp.has_grid = p.chem_mode == 0 ? 1 : 0;
    kp.G = 0;
    for (int a = 0; a < 3; ++a) {
        kp.g[a] = 1;
        kp.inv_h[a] = kp.inv_2h[a] = kp.inv_h2[a] = 0.f;
        kp.hgrid[a] = 0.f;
        kp.hgrid_d[a] = 0.0;
        kp.lo_d[a] = a < p.dim ? p.lo[a] : 0.0;
    }
    kp.pde_bc = p.pde_bc;
    kp.substeps = 1;
    kp.dts = (float)p.dt;
    kp.pde_multi = 0;
    kp.pde_launches = 1;
    kp.zero_src = 0;
    kp.fused_deposit = 0;
    if (!kp.has_grid) return CHEMO_OK;
    int64_t G = 1;
    for (int a = 0; a < p.dim; ++a) {
        kp.g[a] = p.grid[a];
        G *= p.grid[a];
        const double h = grid_h(p, a);
        kp.inv_h[a] = (float)(1.0 / h);
        kp.hgrid[a] = (float)h;
        kp.hgrid_d[a] = h;
        kp.inv_2h[a] = (float)(0.5 / h);
        kp.inv_h2[a] = (float)(1.0 / (h * h));
    }
    if (p.dim == 2) {  // one grid per replicate, stacked as the third index
        kp.g[2] = std::max(kp.layers, 1);
        G *= kp.g[2];
    }
    if (G > ((int64_t)1 << 34)) return fail(CHEMO_EINVAL, "grid too large");
    kp.G = G;
    kp.substeps = resolve_substeps(p);
    kp.dts = (float)(p.dt / kp.substeps);
    // 2D grids with several substeps run them PDE_MULTI_MAX at a time in
    // one launch (the halo of a tile grows by one node per substep)
    kp.pde_multi = (p.dim == 2 && kp.substeps > 1) ? 1 : 0;
    kp.pde_launches = kp.pde_multi ? (kp.substeps + PDE_MULTI_MAX - 1) / PDE_MULTI_MAX : kp.substeps;
    // one substep: the CIC deposit goes straight into c^{n+1} (the density
    // kernel writes a source grid instead)
    kp.fused_deposit = (kp.substeps == 1 && p.pde_bc != 1 && p.deposit_kernel == 0) ? 1 : 0;
    // a CIC deposit into the source grids needs them zero: the next step's
    // particle kernel clears them (a PDE that stored zeros over the values it
    // had just loaded ran at a tenth of the copy rate)
    kp.zero_src = (!kp.fused_deposit && p.deposit_kernel == 0) ? 1 : 0;
    kp.overlap = kp.fused_deposit && p.pde_overlap != 1;
    return CHEMO_OK;
}

int to_status(uint32_t bits)
{
    if (bits & ERR_TIMEOUT) return fail(CHEMO_ETIMEOUT, "a bounded device-side wait ran out (scan look-back)");
    if (bits & ERR_OVERFLOW) return fail(CHEMO_EOVERFLOW, "cell-list placement overflowed");
    if (bits & ERR_NONFINITE) return fail(CHEMO_ENONFINITE, "a non-finite position appeared");
    if (bits & ERR_DOMAIN) return fail(CHEMO_EDOMAIN, "a particle position was outside the box");
    if (bits & ERR_SPECIES) return fail(CHEMO_EINVAL, "a species value was >= n_species");
    return CHEMO_OK;
}

// Kernel parameters with the count buffers of the current parity.
KP view(const chemo_sim *s)
{
    KP k = s->kp;
    k.cnt_cur = s->cnt8[s->cntp];
    k.cnt_nxt = s->cnt8[s->cntp ^ 1];
    return k;
}

// Bins the particles currently in U (with slots already counted into the
// next count buffer) into S.
int sort_from_u(chemo_sim *s, const KP &k, cudaStream_t st)
{
    CUDA_TRY(launch_scan(k, st, nullptr));
    CUDA_TRY(launch_scatter(k, s->cur, 0, st, nullptr));
    s->cntp ^= 1;
    return CHEMO_OK;
}

// The part of a step after the particle kernel: offsets and placement of the
// moved cells (with the CIC deposit, and the step counter advanced), the
// hard-sphere correction with its own re-sort when enabled, and the
// kernel density gather into the source grid when enabled. Flips the count
// buffers once per sort.
int enqueue_sort_and_density(chemo_sim *s, const KP &kp, cudaStream_t st, int *launches)
{
    CUDA_TRY(launch_scan(kp, st, launches));
    CUDA_TRY(launch_scatter(kp, s->cur, kp.hard_sphere ? 0 : 1, st, launches));
    s->cntp ^= 1;
    if (kp.hard_sphere) {
        const KP k2 = view(s);  // S = moved cells, cnt_cur their bins
        CUDA_TRY(launch_hard_sphere(k2, st, launches));
        CUDA_TRY(launch_scan(k2, st, launches));
        CUDA_TRY(launch_scatter(k2, s->cur, 1, st, launches));
        s->cntp ^= 1;
    }
    if (kp.kde && kp.has_grid) CUDA_TRY(launch_kde(view(s), kp.srcg, kp.Rg, st, launches));
    return CHEMO_OK;
}

// Enqueues one step on st. Counts launched kernels into *launches.
int enqueue_step(chemo_sim *s, cudaStream_t st, int *launches)
{
    const KP kp = view(s);
    const bool grid = kp.has_grid && kp.chem_mode == 0;
    const bool overlap = grid && kp.overlap;
    if (grid && kp.fused_deposit && !overlap) CUDA_TRY(launch_pde(kp, s->cur, st, launches));
    if (overlap) {
        // the PDE beside the particle kernels: at the lowest stream priority,
        // so that its blocks take the SMs the pair kernel (the critical path,
        // register-bound at full occupancy) leaves free, and the particle
        // kernels on an internal stream of the highest priority
        CUDA_TRY(cudaEventRecord(s->ev_fork, st));
        CUDA_TRY(cudaStreamWaitEvent(s->aux, s->ev_fork, 0));
        CUDA_TRY(launch_pde(kp, s->cur, s->aux, launches));
        CUDA_TRY(cudaEventRecord(s->ev_join, s->aux));
        CUDA_TRY(cudaStreamWaitEvent(s->hp, s->ev_fork, 0));
        CUDA_TRY(launch_step_particles(kp, s->cur, s->hp, launches));
        CUDA_TRY(cudaEventRecord(s->ev_hp, s->hp));
        CUDA_TRY(cudaStreamWaitEvent(st, s->ev_hp, 0));
        CUDA_TRY(cudaStreamWaitEvent(st, s->ev_join, 0));
    } else {
        CUDA_TRY(launch_step_particles(kp, s->cur, st, launches));
    }
    if (int r = enqueue_sort_and_density(s, kp, st, launches)) return r;
    if (grid && !kp.fused_deposit) CUDA_TRY(launch_pde(kp, s->cur, st, launches));
    if (grid) s->cur = kp.fused_deposit ? (s->cur ^ 1) : (s->cur ^ (kp.pde_launches & 1));
    s->step += 1;
    return CHEMO_OK;
}

void drop_graphs(chemo_sim *s)
{
    for (auto &a : s->graph)
        for (auto &b : a)
            for (auto &g : b)
                if (g) {
                    cudaGraphExecDestroy(g);
                    g = nullptr;
                }
}

// Captures `k` steps starting from the current buffer parities into an
// executable graph (the parities are restored afterwards).
int capture(chemo_sim *s, int k, cudaGraphExec_t *out)
{
    const int cur0 = s->cur, cntp0 = s->cntp;
    const int64_t step0 = s->step;
    CUDA_TRY(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    int st = CHEMO_OK;
    for (int i = 0; i < k && st == CHEMO_OK; ++i) st = enqueue_step(s, s->cap, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->cap, &g);
    s->cur = cur0;
    s->cntp = cntp0;
    s->step = step0;
    if (st != CHEMO_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(CHEMO_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    // the kernel nodes keep the priorities of the streams they were captured on
    e = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(CHEMO_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return CHEMO_OK;
}

int copy_in(chemo_sim *s, const void *src, size_t bytes, int mem_kind, cudaStream_t st, size_t offset, void **dst)
{
    if (mem_kind == CHEMO_MEM_DEVICE) {
        *dst = const_cast<void *>(src);
        return CHEMO_OK;
    }
    (void)s;
    char *base = (char *)s->scratch + offset;
    CUDA_TRY(cudaMemcpyAsync(base, src, bytes, cudaMemcpyHostToDevice, st));
    *dst = base;
    return CHEMO_OK;
}

int check_mem_kind(int mem_kind)
{
    if (mem_kind != CHEMO_MEM_HOST && mem_kind != CHEMO_MEM_DEVICE)
        return fail(CHEMO_EINVAL, "mem_kind must be CHEMO_MEM_HOST (0) or CHEMO_MEM_DEVICE (1)");
    return CHEMO_OK;
}

int ingest(chemo_sim *s, const float *pos, const uint8_t *sp, const float *disp, int mem_kind, cudaStream_t st)
{
    const int64_t n = s->kp.n;
    const int d = s->kp.dim;
    if (n == 0) return sort_from_u(s, view(s), st);
    if (!pos || !sp) return fail(CHEMO_EINVAL, "pos and species are required");
    // positions and species are validated by the pack kernel on the device;
    // bad entries are clamped and latched (reported by chemo_check)
    const size_t pbytes = (size_t)n * d * sizeof(float);
    const size_t sbytes = ((size_t)n + 255) & ~(size_t)255;
    if (mem_kind == CHEMO_MEM_HOST) {
        void *tmp = nullptr;
        int r = scratch(s, 2 * pbytes + sbytes + 512, &tmp);
        if (r) return r;
    }
    void *dpos = nullptr, *dsp = nullptr, *ddisp = nullptr;
    int r = copy_in(s, pos, pbytes, mem_kind, st, 0, &dpos);
    if (r) return r;
    r = copy_in(s, sp, (size_t)n, mem_kind, st, (pbytes + 255) & ~(size_t)255, &dsp);
    if (r) return r;
    if (disp && s->kp.dS) {
        r = copy_in(s, disp, pbytes, mem_kind, st, ((pbytes + 255) & ~(size_t)255) + sbytes, &ddisp);
        if (r) return r;
    }
    const KP k = view(s);
    CUDA_TRY(launch_pack(k, (const float *)dpos, (const uint8_t *)dsp, (const float *)ddisp, st, nullptr));
    r = sort_from_u(s, k, st);
    if (r) return r;
    if (mem_kind == CHEMO_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(st));
    return CHEMO_OK;
}

}  // namespace

int eng_fail(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return status;
}
int eng_dalloc(chemo_sim *s, void **p, size_t bytes) { return dalloc(s, p, bytes); }

DevMem eng_allocator()
{
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    return g_alloc;
}

int eng_mem_alloc(const DevMem &m, void **p, size_t bytes, size_t *rounded)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (rounded) *rounded = bytes;
    if (m.alloc) {
        void *q = nullptr;
        const int rc = m.alloc(m.ctx, bytes, &q);
        if (rc != 0 || !q)
            return fail(CHEMO_ENOMEM, "the allocator given to chemo_set_allocator failed for %zu bytes (status %d)",
                        bytes, rc);
        if (reinterpret_cast<uintptr_t>(q) & 255u) {
            m.release(m.ctx, q, bytes);
            return fail(CHEMO_ENOMEM, "the allocator given to chemo_set_allocator returned a pointer not aligned "
                                      "to 256 bytes");
        }
        *p = q;
        return CHEMO_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(CHEMO_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    return CHEMO_OK;
}

void eng_mem_release(const DevMem &m, void *p, size_t bytes)
{
    if (!p) return;
    if (m.release)
        m.release(m.ctx, p, bytes);
    else
        cudaFree(p);
}

int chemo_set_allocator(chemo_alloc_fn alloc, chemo_release_fn release, void *ctx)
{
    g_last_error[0] = 0;
    if ((alloc == nullptr) != (release == nullptr))
        return fail(CHEMO_EINVAL, "alloc and release are both set or both NULL");
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return CHEMO_OK;
}
int eng_scratch(chemo_sim *s, size_t bytes, void **p) { return scratch(s, bytes, p); }
KP eng_view(const chemo_sim *s) { return view(s); }
int eng_enqueue_step(chemo_sim *s, cudaStream_t st, int *launches) { return enqueue_step(s, st, launches); }
int eng_ingest(chemo_sim *s, const float *pos, const uint8_t *sp, const float *disp, int mem_kind, cudaStream_t st)
{
    return ingest(s, pos, sp, disp, mem_kind, st);
}
void eng_drop_graphs(chemo_sim *s) { drop_graphs(s); }
void eng_fill_model(const chemo_params &p, KP &kp) { fill_model(p, kp); }

// Parameter block of a particle set that is binned and searched only
// (no grid, no buffers): validation, cell-list layout and model constants.
int chemo_internal_build_kp(const chemo_params *params, int64_t n, KP *out)
{
    g_last_error[0] = 0;
    if (!params || !out) return fail(CHEMO_EINVAL, "params and out are required");
    if (int r = check_params(*params)) return r;
    if (n < 0 || n > (int64_t)ID_MASK + 1) return fail(CHEMO_EINVAL, "n = %lld out of range", (long long)n);
    KP kp{};
    kp.n = n;
    kp.layers = 1;
    kp.layer_off = nullptr;
    if (int r = fill_layout(*params, n, kp)) return r;
    if (int r = fill_grid(*params, kp)) return r;
    fill_model(*params, kp);
    *out = kp;
    return CHEMO_OK;
}

int chemo_internal_fail(int status, const char *msg) { return fail(status, "%s", msg); }

extern "C" {

const char *chemo_status_string(int status)
{
    switch (status) {
    case CHEMO_OK: return "ok";
    case CHEMO_EINVAL: return "invalid argument";
    case CHEMO_ENOMEM: return "out of memory";
    case CHEMO_ECUDA: return "CUDA error";
    case CHEMO_EDOMAIN: return "particle outside the domain";
    case CHEMO_ENONFINITE: return "non-finite value";
    case CHEMO_EOVERFLOW: return "overflow";
    case CHEMO_ETIMEOUT: return "device wait timed out";
    case CHEMO_ENOTSUP: return "not supported";
    default: return "unknown status";
    }
}

const char *chemo_last_error(void) { return g_last_error; }

void chemo_destroy(chemo_sim *s)
{
    if (!s) return;
    cudaDeviceSynchronize();
    drop_graphs(s);
    chemo_tape_free(s->tape);
    for (const DevBuf &b : s->allocs) eng_mem_release(s->mem, b.ptr, b.bytes);
    eng_mem_release(s->mem, s->scratch, s->scratch_bytes);
    if (s->aux) cudaStreamDestroy(s->aux);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_hp) cudaEventDestroy(s->ev_hp);
    if (s->hp) cudaStreamDestroy(s->hp);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    delete s;
}

int chemo_create(const chemo_params *params, int64_t n, const float *pos, const uint8_t *species, int mem_kind,
                 void *stream, chemo_sim **out)
{
    ChemoRange nvtx_range("chemo_create");
    return chemo_create_batch(params, 1, &n, pos, species, mem_kind, stream, out);
}

}  // extern "C"

namespace {

// A sub-domain keeps every deposit in the source grids and runs its PDE
// after the particle part on one stream (the halo planes of the source are
// exchanged in between).
void apply_subdomain(KP &kp, uint32_t open_faces)
{
    kp.sub = 1;
    kp.open_z = (int)open_faces;
    kp.fused_deposit = 0;
    kp.overlap = 0;
    kp.zero_src = 1;
}

int launches_per_step(const KP &kp)
{
    const int64_t n = kp.n;
    return (n > 0 ? (kp.pairs && kp.search == 4 ? 2 : 1) : 0) + 2 + (kp.has_grid ? kp.pde_launches : 0) +
           (kp.hard_sphere ? (n > 0 ? 3 : 2) : 0) + (kp.kde && kp.has_grid ? 1 : 0);
}

// Creates a simulation of `replicates` layers holding off[replicates] cells
// (buffers for `capacity` >= that many); a sub-domain when sub.
int create_sim(const chemo_params *params, int32_t replicates, const std::vector<int64_t> &off, int64_t capacity,
               bool sub, uint32_t open_faces, const float *pos, const uint8_t *species, int mem_kind,
               cudaStream_t st, chemo_sim **out)
{
    const int64_t n = off[(size_t)replicates];
    chemo_sim *s = new (std::nothrow) chemo_sim();
    if (!s) return fail(CHEMO_ENOMEM, "host allocation failed");
    s->mem = eng_allocator();
    s->prm = *params;
    s->capacity = capacity;
    KP &kp = s->kp;
    kp.n = n;
    kp.layers = replicates;
    kp.layer_off = nullptr;
    kp.sub = 0;
    kp.open_z = 0;
    s->layer_off_host = off;
    int r;
    if ((r = fill_layout(*params, capacity, kp)) || (r = fill_grid(*params, kp))) {
        delete s;
        return r;
    }
    if (sub) apply_subdomain(kp, open_faces);
    fill_model(*params, kp);
    const size_t N = (size_t)std::max<int64_t>(capacity, 1);
    void *p;
#define ALLOC(field, bytes)                         \
    if ((r = dalloc(s, &p, (bytes)))) {             \
        chemo_destroy(s);                           \
        return r;                                   \
    }                                               \
    field = decltype(field)(p);
    ALLOC(kp.S, N * sizeof(float4));
    ALLOC(kp.U, N * sizeof(float4));
    ALLOC(kp.slot, N * sizeof(uint32_t));
    kp.Fh = nullptr;
    if (kp.pairs && kp.search == 4) {  // half-window force sums, cleared by each step's particle kernel
        const size_t fb = N * (size_t)(kp.dim == 3 ? 4 : 2) * sizeof(long long);
        ALLOC(kp.Fh, fb);
        if (cudaMemsetAsync(kp.Fh, 0, fb, st) != cudaSuccess) {
            chemo_destroy(s);
            return fail(CHEMO_ECUDA, "create: clearing the force sums failed");
        }
    }
    kp.dS = kp.dU = nullptr;
    if (params->track_displacement) {
        ALLOC(kp.dS, N * sizeof(float4));
        ALLOC(kp.dU, N * sizeof(float4));
    }
    const size_t slots = (size_t)kp.bin_slots;  // a multiple of 8
    const size_t cwords = slots / 2;  // 16-bit counts
    ALLOC(s->cnt8[0], cwords * sizeof(uint32_t));
    ALLOC(s->cnt8[1], cwords * sizeof(uint32_t));
    ALLOC(kp.gstart, (((size_t)kp.ngroups + 1 + 3) & ~(size_t)3) * sizeof(uint32_t));
    kp.cnt_cur = kp.cnt_nxt = nullptr;
    const size_t tiles = ((size_t)kp.ngroups + 2047) / 2048;
    ALLOC(kp.tiles, tiles * sizeof(unsigned long long));
    uint32_t *ctl;
    ALLOC(ctl, 64);
    kp.tile_ctr = ctl;
    kp.scan_seq = ctl + 1;
    kp.err = ctl + 2;
    kp.step = reinterpret_cast<unsigned long long *>(ctl + 4);
    kp.pair_count = nullptr;  // set only while profiling
    kp.test_count = nullptr;
    if (replicates > 1) {
        int64_t *lo;
        ALLOC(lo, off.size() * sizeof(int64_t));
        kp.layer_off = lo;
    }
    kp.c[0] = kp.c[1] = nullptr;
    kp.srcg = kp.Rg = nullptr;
    if (kp.has_grid) {
        ALLOC(kp.c[0], (size_t)kp.G * sizeof(float));
        ALLOC(kp.c[1], (size_t)kp.G * sizeof(float));
        if (!kp.fused_deposit) {
            ALLOC(kp.srcg, (size_t)kp.G * sizeof(float));
            ALLOC(kp.Rg, (size_t)kp.G * sizeof(float));
        }
    }
#undef ALLOC
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemsetAsync(s->cnt8[0], 0, cwords * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->cnt8[1], 0, cwords * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(kp.tiles, 0, tiles * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, 64, st);
    if (e == cudaSuccess && kp.layer_off)  // from the simulation's own host copy (outlives the copy)
        e = cudaMemcpyAsync(const_cast<int64_t *>(kp.layer_off), s->layer_off_host.data(),
                            s->layer_off_host.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && kp.has_grid) {
        e = cudaMemsetAsync(kp.c[0], 0, (size_t)kp.G * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(kp.c[1], 0, (size_t)kp.G * sizeof(float), st);
        if (e == cudaSuccess && kp.srcg) e = cudaMemsetAsync(kp.srcg, 0, (size_t)kp.G * sizeof(float), st);
        if (e == cudaSuccess && kp.Rg) e = cudaMemsetAsync(kp.Rg, 0, (size_t)kp.G * sizeof(float), st);
    }
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->aux, cudaStreamNonBlocking, prio_lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->hp, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_hp, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        chemo_destroy(s);
        return fail(CHEMO_ECUDA, "create: %s", cudaGetErrorString(e));
    }
    if ((r = ingest(s, pos, species, nullptr, mem_kind, st))) {
        chemo_destroy(s);
        return r;
    }
    // launches per step: particles, scan, scatter, and the PDE substeps
    s->launches_per_step = launches_per_step(kp);
    *out = s;
    return CHEMO_OK;
}

}  // namespace

extern "C" {

int chemo_create_batch(const chemo_params *params, int32_t replicates, const int64_t *n_per_replicate,
                       const float *pos, const uint8_t *species, int mem_kind, void *stream, chemo_sim **out)
{
    ChemoRange nvtx_range("chemo_create_batch");
    g_last_error[0] = 0;
    if (!params || !out || !n_per_replicate) return fail(CHEMO_EINVAL, "params, n_per_replicate and out are required");
    *out = nullptr;
    if (int r = check_mem_kind(mem_kind)) return r;
    if (int r = check_params(*params)) return r;
    if (replicates < 1 || replicates > 65535) return fail(CHEMO_EINVAL, "replicates = %d out of range [1, 65535]", replicates);
    if (replicates > 1 && params->dim != 2) return fail(CHEMO_EINVAL, "replicates > 1 needs dim = 2");
    std::vector<int64_t> off((size_t)replicates + 1, 0);
    for (int r = 0; r < replicates; ++r) {
        const int64_t m = n_per_replicate[r];
        if (m < 0 || m > (int64_t)ID_MASK + 1) return fail(CHEMO_EINVAL, "replicate %d: n = %lld out of range", r, (long long)m);
        off[(size_t)r + 1] = off[(size_t)r] + m;
        if (off[(size_t)r + 1] > (int64_t)ID_MASK + 1) return fail(CHEMO_EINVAL, "more than 2^29 cells in total");
    }
    const int64_t n = off[(size_t)replicates];
    if (n > 0 && mem_kind == CHEMO_MEM_DEVICE && !(is_device_ptr(pos) && is_device_ptr(species)))
        return fail(CHEMO_EINVAL, "mem_kind is DEVICE but pos/species are not device pointers");
    return create_sim(params, replicates, off, n, false, 0u, pos, species, mem_kind, (cudaStream_t)stream, out);
}

int chemo_create_subdomain(const chemo_params *params, int64_t capacity, uint32_t open_faces, void *stream,
                           chemo_sim **out)
{
    ChemoRange nvtx_range("chemo_create_subdomain");
    g_last_error[0] = 0;
    if (!params || !out) return fail(CHEMO_EINVAL, "params and out are required");
    *out = nullptr;
    if (int r = check_params(*params)) return r;
    const chemo_params &p = *params;
    if (p.dim != 3) return fail(CHEMO_EINVAL, "sub-domains are z-slabs of a 3D system (dim = %d)", p.dim);
    if (p.boundary != 0 || p.chem_mode != 0)
        return fail(CHEMO_ENOTSUP, "sub-domains need reflecting walls (boundary 0) and the grid (chem_mode 0)");
    if (p.hard_sphere || p.deposit_kernel != 0)
        return fail(CHEMO_ENOTSUP, "sub-domains support neither hard_sphere nor deposit_kernel 1");
    if (capacity < 1 || capacity > (int64_t)ID_MASK)
        return fail(CHEMO_EINVAL, "capacity = %lld out of range [1, 2^29 - 1]", (long long)capacity);
    if (open_faces > (CHEMO_OPEN_ZLO | CHEMO_OPEN_ZHI)) return fail(CHEMO_EINVAL, "open_faces = %u: bits 0 and 1 only", open_faces);
    const std::vector<int64_t> off(2, 0);
    return create_sim(params, 1, off, capacity, true, open_faces, nullptr, nullptr, CHEMO_MEM_DEVICE,
                      (cudaStream_t)stream, out);
}

static int need_subdomain(const chemo_sim *s, const char *what)
{
    if (!s) return fail(CHEMO_EINVAL, "sim is NULL");
    if (!s->kp.sub) return fail(CHEMO_ENOTSUP, "%s: not a sub-domain (chemo_create_subdomain)", what);
    return CHEMO_OK;
}

int chemo_slab_ingest(chemo_sim *s, int64_t n, const chemo_cell *cells, int mem_kind, void *stream)
{
    ChemoRange nvtx_range("chemo_slab_ingest");
    g_last_error[0] = 0;
    if (int r = need_subdomain(s, "chemo_slab_ingest")) return r;
    if (int r = check_mem_kind(mem_kind)) return r;
    if (n < 0 || n > s->capacity)
        return fail(CHEMO_EINVAL, "n = %lld out of range [0, capacity = %lld]", (long long)n, (long long)s->capacity);
    if (n > 0 && !cells) return fail(CHEMO_EINVAL, "cells is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)n * sizeof(chemo_cell);
    const float4 *rec = reinterpret_cast<const float4 *>(cells);
    if (n > 0 && mem_kind == CHEMO_MEM_DEVICE) {
        if (((uintptr_t)cells & 15u) != 0) return fail(CHEMO_EINVAL, "cells must be 16-byte aligned");
        if (!is_device_ptr(cells)) return fail(CHEMO_EINVAL, "mem_kind is DEVICE but cells is not a device pointer");
    } else if (n > 0) {
        void *tmp = nullptr;
        if (int r = scratch(s, bytes, &tmp)) return r;
        CUDA_TRY(cudaMemcpyAsync(tmp, cells, bytes, cudaMemcpyHostToDevice, st));
        rec = static_cast<const float4 *>(tmp);
    }
    if (n != s->kp.n) {
        drop_graphs(s);  // graphs hold the old count
        s->kp.n = n;
        s->launches_per_step = launches_per_step(s->kp);
    }
    const KP k = view(s);
    CUDA_TRY(launch_pack_cells(k, rec, st));
    if (int r = sort_from_u(s, k, st)) return r;
    if (mem_kind == CHEMO_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(st));
    return CHEMO_OK;
}

int chemo_slab_select(chemo_sim *s, int32_t ntargets, const chemo_slab_target *targets, void *stream)
{
    g_last_error[0] = 0;
    if (int r = need_subdomain(s, "chemo_slab_select")) return r;
    if (ntargets < 0 || ntargets > SLAB_TARGETS) return fail(CHEMO_EINVAL, "ntargets = %d out of range [0, %d]", ntargets, SLAB_TARGETS);
    if (ntargets > 0 && !targets) return fail(CHEMO_EINVAL, "targets is NULL");
    SlabSelect t{};
    t.nt = ntargets;
    for (int k = 0; k < ntargets; ++k) {
        const chemo_slab_target &g = targets[k];
        if (g.capacity < 0) return fail(CHEMO_EINVAL, "target %d: negative capacity", k);
        if (g.capacity > 0 && (!g.out || ((uintptr_t)g.out & 15u) != 0))
            return fail(CHEMO_EINVAL, "target %d: out must be a 16-byte aligned device array", k);
        if (!g.count || ((uintptr_t)g.count & 7u) != 0) return fail(CHEMO_EINVAL, "target %d: count must be an aligned device pointer", k);
        t.z0[k] = g.z0;
        t.z1[k] = g.z1;
        t.own0[k] = g.own0;
        t.own1[k] = g.own1;
        t.out[k] = reinterpret_cast<float4 *>(g.out);
        t.cap[k] = g.capacity;
        t.count[k] = g.count;
    }
    CUDA_TRY(launch_slab_select(view(s), t, (cudaStream_t)stream));
    return CHEMO_OK;
}

int chemo_slab_planes(chemo_sim *s, int32_t grid, int32_t op, int64_t plane0, int64_t nplanes, float *buf,
                      void *stream)
{
    g_last_error[0] = 0;
    if (int r = need_subdomain(s, "chemo_slab_planes")) return r;
    const KP &kp = s->kp;
    if (grid < 0 || grid > 2) return fail(CHEMO_EINVAL, "grid = %d: 0 (c), 1 (source) or 2 (consumption)", grid);
    if (op < CHEMO_PLANES_READ || op > CHEMO_PLANES_ADD) return fail(CHEMO_EINVAL, "op = %d: 0 read, 1 write, 2 add", op);
    if (plane0 < 0 || nplanes < 0 || plane0 + nplanes > kp.g[2])
        return fail(CHEMO_EINVAL, "planes [%lld, %lld) outside [0, %d)", (long long)plane0, (long long)(plane0 + nplanes), kp.g[2]);
    if (nplanes == 0) return CHEMO_OK;
    if (!buf) return fail(CHEMO_EINVAL, "buf is NULL");
    const int64_t P = (int64_t)kp.g[0] * kp.g[1];
    float *base = grid == 0 ? kp.c[s->cur] : (grid == 1 ? kp.srcg : kp.Rg);
    float *g = base + plane0 * P;
    const int64_t m = nplanes * P;
    cudaStream_t st = (cudaStream_t)stream;
    if (op == CHEMO_PLANES_READ) CUDA_TRY(cudaMemcpyAsync(buf, g, (size_t)m * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else if (op == CHEMO_PLANES_WRITE) CUDA_TRY(cudaMemcpyAsync(g, buf, (size_t)m * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else CUDA_TRY(launch_add(g, buf, m, st));
    return CHEMO_OK;
}

int chemo_step_particles(chemo_sim *s, void *stream)
{
    ChemoRange nvtx_range("chemo_step_particles");
    g_last_error[0] = 0;
    if (int r = need_subdomain(s, "chemo_step_particles")) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const KP kp = view(s);
    CUDA_TRY(launch_step_particles(kp, s->cur, st, nullptr));
    if (int r = enqueue_sort_and_density(s, kp, st, nullptr)) return r;
    s->step += 1;
    return CHEMO_OK;
}

int chemo_step_field(chemo_sim *s, void *stream)
{
    ChemoRange nvtx_range("chemo_step_field");
    g_last_error[0] = 0;
    if (int r = need_subdomain(s, "chemo_step_field")) return r;
    const KP kp = view(s);
    CUDA_TRY(launch_pde(kp, s->cur, (cudaStream_t)stream, nullptr));
    s->cur ^= (kp.pde_launches & 1);
    return CHEMO_OK;
}

// Device time per step of one candidate parameter set (ms), or a status.
static int trial_time(const chemo_params &q, int32_t replicates, const int64_t *n_per, const float *pos,
                      const uint8_t *species, int mem_kind, int32_t trial_steps, cudaStream_t st, float *ms)
{
    chemo_sim *sim = nullptr;
    int r = chemo_create_batch(&q, replicates, n_per, pos, species, mem_kind, st, &sim);
    if (r) return r;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        r = chemo_step_n(sim, 4, st);  // warm-up (captures the graphs)
        if (!r) e = cudaEventRecord(e0, st);
        if (!r && e == cudaSuccess) r = chemo_step_n(sim, trial_steps, st);
        if (!r && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (!r && e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (!r && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        if (!r && e == cudaSuccess) {
            *ms /= (float)trial_steps;
            r = chemo_check(sim, st);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    chemo_destroy(sim);
    if (!r && e != cudaSuccess) r = fail(CHEMO_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
    return r;
}

int chemo_autotune(const chemo_params *params, int32_t replicates, const int64_t *n_per_replicate,
                   const float *pos, const uint8_t *species, int mem_kind, int32_t trial_steps, void *stream,
                   chemo_params *best_out, float *best_ms_out)
{
    ChemoRange nvtx_range("chemo_autotune");
    g_last_error[0] = 0;
    if (!params || !best_out || !n_per_replicate) return fail(CHEMO_EINVAL, "params, n_per_replicate and best_out are required");
    if (trial_steps < 1) return fail(CHEMO_EINVAL, "trial_steps must be >= 1");
    if (int r = check_params(*params)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const double rc = max_cutoff(*params);
    std::vector<chemo_params> cands;
    if (rc > 0.0 && params->inter != 0.f) {
        // bin side factors of each search mode (1: 3^d warp, 2: 2^d, 3: 3^d per
        // lane, 4: half of the 3^d window per lane)
        const double fac[4][4] = {{1.0, 1.25, 1.5, 2.0}, {1.0, 1.25, 0.0, 0.0}, {1.0, 1.5, 0.0, 0.0}, {1.0, 1.25, 1.5, 0.0}};
        const int nf[4] = {4, 2, 2, 3};
        for (int mode = 1; mode <= 4; ++mode) {
            const double bmin = (mode == 2 ? 2.0 : 1.0) * rc * (1.0 + 1.0 / 4096.0);
            for (int k = 0; k < nf[mode - 1]; ++k) {
                chemo_params q = *params;
                q.search_mode = mode;
                // the minimum side is the automatic one; larger sides are well above it
                q.bin_side = k == 0 ? 0.f : (float)(bmin * fac[mode - 1][k]);
                cands.push_back(q);
            }
        }
    } else {
        cands.push_back(*params);
    }
    int best = -1;
    float best_ms = 0.f;
    int last_err = CHEMO_OK;
    for (size_t i = 0; i < cands.size(); ++i) {
        float ms = 0.f;
        const int r = trial_time(cands[i], replicates, n_per_replicate, pos, species, mem_kind, trial_steps, st, &ms);
        if (r == CHEMO_EINVAL) {  // layout not admissible for this box (too few periodic bins...)
            last_err = r;
            continue;
        }
        if (r) return r;
        if (best < 0 || ms < best_ms) {
            best = (int)i;
            best_ms = ms;
        }
    }
    if (best < 0) return last_err ? last_err : fail(CHEMO_EINVAL, "no admissible candidate");
    chemo_params q = cands[(size_t)best];
    if (q.search_mode == 1) {  // how sparse a warp may be and still search together
        const int runs[3] = {4, 8, 32};
        for (int v : runs) {
            chemo_params c = q;
            c.warp_runs = v;
            float ms = 0.f;
            const int r = trial_time(c, replicates, n_per_replicate, pos, species, mem_kind, trial_steps, st, &ms);
            if (r) return r;
            if (ms < best_ms) {
                best_ms = ms;
                q = c;
            }
        }
    }
    if ((q.search_mode == 0 || q.search_mode == 4) && rc > 0.0 && params->inter != 0.f) {
        // threads per block of the half-window pair and move kernels
        const int bts[2] = {128, 512};
        for (int b : bts) {
            chemo_params c = q;
            c.block_threads = b;
            float ms = 0.f;
            const int r = trial_time(c, replicates, n_per_replicate, pos, species, mem_kind, trial_steps, st, &ms);
            if (r) return r;
            if (ms < best_ms) {
                best_ms = ms;
                q = c;
            }
        }
    }
    if (params->chem_mode == 0) {  // PDE overlap (one-substep fields): try the other settings
        for (int ov = 1; ov <= 2; ++ov) {
            chemo_params v = q;
            v.pde_overlap = ov;
            float ms = 0.f;
            const int r = trial_time(v, replicates, n_per_replicate, pos, species, mem_kind, trial_steps, st, &ms);
            if (r) return r;
            if (ms < best_ms) {
                best_ms = ms;
                q = v;
            }
        }
    }
    g_last_error[0] = 0;
    *best_out = q;
    if (best_ms_out) *best_ms_out = best_ms;
    return CHEMO_OK;
}

int chemo_write_state(chemo_sim *s, const float *pos, const uint8_t *species, const float *disp, int mem_kind,
                      void *stream)
{
    ChemoRange nvtx_range("chemo_write_state");
    g_last_error[0] = 0;
    if (s && s->kp.sub) return fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_write_state");
    if (!s) return fail(CHEMO_EINVAL, "sim is NULL");
    if (int r = check_mem_kind(mem_kind)) return r;
    return ingest(s, pos, species, disp, mem_kind, (cudaStream_t)stream);
}

int chemo_write_field(chemo_sim *s, const float *c, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    if (!s || !c) return fail(CHEMO_EINVAL, "sim and c are required");
    if (int r = check_mem_kind(mem_kind)) return r;
    if (!s->kp.has_grid) return fail(CHEMO_EINVAL, "this simulation has no grid (chem_mode 1)");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)s->kp.G * sizeof(float);
    CUDA_TRY(cudaMemcpyAsync(s->kp.c[s->cur], c, bytes,
                             mem_kind == CHEMO_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    if (mem_kind == CHEMO_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(st));
    return CHEMO_OK;
}

int chemo_step(chemo_sim *s, void *stream)
{
    ChemoRange nvtx_range("chemo_step");
    g_last_error[0] = 0;
    if (!s) return fail(CHEMO_EINVAL, "sim is NULL");
    return enqueue_step(s, (cudaStream_t)stream, nullptr);
}

int chemo_step_n(chemo_sim *s, int64_t nsteps, void *stream)
{
    ChemoRange nvtx_range("chemo_step_n");
    g_last_error[0] = 0;
    if (!s) return fail(CHEMO_EINVAL, "sim is NULL");
    if (nsteps < 0) return fail(CHEMO_EINVAL, "nsteps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t left = nsteps;
    // graphs of an even number of steps leave both buffer parities unchanged
    static const int sizes[2] = {2, 16};
    for (int gi = 1; gi >= 0; --gi) {
        const int k = sizes[gi];
        if (left < k) continue;
        cudaGraphExec_t &g = s->graph[gi][s->cur][s->cntp];
        if (!g) {
            // capture this size for every buffer parity at once, so that later
            // calls (after a chemo_write_state, for instance) never capture
            const int cur0 = s->cur, cntp0 = s->cntp;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    if (s->graph[gi][a][b]) continue;
                    s->cur = a;
                    s->cntp = b;
                    const int r = capture(s, k, &s->graph[gi][a][b]);
                    s->cur = cur0;
                    s->cntp = cntp0;
                    if (r) return r;
                }
        }
        while (left >= k) {
            CUDA_TRY(cudaGraphLaunch(g, st));
            s->step += k;
            left -= k;
        }
    }
    while (left > 0) {
        if (int r = enqueue_step(s, st, nullptr)) return r;
        --left;
    }
    return CHEMO_OK;
}

int chemo_read_state(chemo_sim *s, float *pos_out, uint8_t *species_out, float *disp_out, int mem_kind, void *stream)
{
    ChemoRange nvtx_range("chemo_read_state");
    g_last_error[0] = 0;
    if (s && s->kp.sub) return fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_read_state");
    if (!s) return fail(CHEMO_EINVAL, "sim is NULL");
    if (int r = check_mem_kind(mem_kind)) return r;
    if (disp_out && !s->kp.dS) return fail(CHEMO_EINVAL, "displacement is not tracked (track_displacement = 0)");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = s->kp.n;
    const size_t pbytes = (size_t)n * s->kp.dim * sizeof(float);
    const size_t pb = (pbytes + 255) & ~(size_t)255;
    if (mem_kind == CHEMO_MEM_DEVICE) {
        CUDA_TRY(launch_unsort(view(s), pos_out, species_out, disp_out, st));
    } else {
        void *tmp = nullptr;
        if (int r = scratch(s, 2 * pb + (size_t)n + 256, &tmp)) return r;
        char *b = (char *)tmp;
        float *dp = pos_out ? (float *)b : nullptr;
        float *dd = disp_out ? (float *)(b + pb) : nullptr;
        uint8_t *ds = species_out ? (uint8_t *)(b + 2 * pb) : nullptr;
        CUDA_TRY(launch_unsort(view(s), dp, ds, dd, st));
        if (pos_out && n) CUDA_TRY(cudaMemcpyAsync(pos_out, dp, pbytes, cudaMemcpyDeviceToHost, st));
        if (disp_out && n) CUDA_TRY(cudaMemcpyAsync(disp_out, dd, pbytes, cudaMemcpyDeviceToHost, st));
        if (species_out && n) CUDA_TRY(cudaMemcpyAsync(species_out, ds, (size_t)n, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return chemo_check(s, stream);
    }
    return CHEMO_OK;
}

int chemo_read_field(chemo_sim *s, float *c_out, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    if (!s || !c_out) return fail(CHEMO_EINVAL, "sim and c_out are required");
    if (int r = check_mem_kind(mem_kind)) return r;
    if (!s->kp.has_grid) return fail(CHEMO_EINVAL, "this simulation has no grid (chem_mode 1)");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(c_out, s->kp.c[s->cur], (size_t)s->kp.G * sizeof(float),
                             mem_kind == CHEMO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    if (mem_kind == CHEMO_MEM_HOST) {
        CUDA_TRY(cudaStreamSynchronize(st));
        return chemo_check(s, stream);
    }
    return CHEMO_OK;
}

int chemo_set_params(chemo_sim *s, const chemo_params *p)
{
    g_last_error[0] = 0;
    if (!s || !p) return fail(CHEMO_EINVAL, "sim and params are required");
    if (int r = check_params(*p)) return r;
    const chemo_params &o = s->prm;
    bool same = p->dim == o.dim && p->boundary == o.boundary && p->n_species == o.n_species &&
                p->chem_mode == o.chem_mode && p->pde_bc == o.pde_bc && p->track_displacement == o.track_displacement;
    for (int a = 0; a < 3; ++a) same = same && p->lo[a] == o.lo[a] && p->hi[a] == o.hi[a] && p->grid[a] == o.grid[a];
    if (!same) return fail(CHEMO_EINVAL, "chemo_set_params cannot change geometry, species count or modes");
    KP k2 = s->kp;
    int r;
    if ((r = fill_layout(*p, s->capacity, k2)) || (r = fill_grid(*p, k2))) return r;
    if (s->kp.sub) apply_subdomain(k2, (uint32_t)s->kp.open_z);
    if (k2.nb[0] != s->kp.nb[0] || k2.nb[1] != s->kp.nb[1] || k2.nb[2] != s->kp.nb[2] ||
        k2.search != s->kp.search || k2.px != s->kp.px || k2.substeps != s->kp.substeps ||
        k2.fused_deposit != s->kp.fused_deposit || k2.overlap != s->kp.overlap)
        return fail(CHEMO_EINVAL, "new parameters change the cell-list layout or the PDE substeps");
    fill_model(*p, s->kp);
    s->prm = *p;
    drop_graphs(s);  // graphs hold the old constants
    chemo_tape_free(s->tape);  // a recorded run belongs to the old parameters
    s->tape = nullptr;
    return CHEMO_OK;
}

int64_t chemo_step_index(const chemo_sim *s) { return s ? s->step : -1; }

int chemo_set_step_index(chemo_sim *s, int64_t step, void *stream)
{
    g_last_error[0] = 0;
    if (!s || step < 0) return fail(CHEMO_EINVAL, "bad sim or step");
    k_set_u64<<<1, 1, 0, (cudaStream_t)stream>>>(s->kp.step, (unsigned long long)step);
    CUDA_TRY(cudaGetLastError());
    s->step = step;
    return CHEMO_OK;
}

int chemo_check(chemo_sim *s, void *stream)
{
    if (!s) return fail(CHEMO_EINVAL, "sim is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaStreamSynchronize(s->aux));
    uint32_t bits = 0;
    CUDA_TRY(cudaMemcpy(&bits, s->kp.err, sizeof(bits), cudaMemcpyDeviceToHost));
    if (bits) CUDA_TRY(cudaMemset(s->kp.err, 0, sizeof(uint32_t)));
    return to_status(bits);
}

int chemo_get_info(const chemo_sim *s, chemo_info *info)
{
    if (!s || !info) return fail(CHEMO_EINVAL, "sim and info are required");
    const KP &kp = s->kp;
    info->n = kp.n;
    info->dim = kp.dim;
    info->search_mode = kp.search;
    for (int a = 0; a < 3; ++a) {
        info->nbins[a] = kp.nb[a];
        info->bin_side[a] = a < kp.dim ? kp.L[a] / kp.nb[a] : 0.f;
    }
    info->bin_slots = kp.bin_slots;
    info->bin_pitch = kp.px;
    info->pde_substeps = kp.has_grid ? kp.substeps : 0;
    info->grid_nodes = kp.G;
    info->device_bytes = s->bytes;
    info->launches_per_step = s->launches_per_step;
    info->layers = kp.layers;
    // the paper's rule of thumb for the time step against the interaction range
    const chemo_params &p = s->prm;
    double ratio = 0.0;
    for (int a = 0; a < p.n_species; ++a)
        for (int b = 0; b < p.n_species; ++b) {
            const double eps = 0.5 * ((double)p.diameter[a] + (double)p.diameter[b]);
            if (eps > 0.0) ratio = std::max(ratio, std::sqrt(2.0 * ((double)p.D[a] + (double)p.D[b]) * p.dt) / eps);
        }
    info->step_ratio = (float)ratio;
    return CHEMO_OK;
}

int chemo_profile_steps(chemo_sim *s, int64_t nsteps, float *kernel_ms, void *stream)
{
    ChemoRange nvtx_range("chemo_profile_steps");
    g_last_error[0] = 0;
    if (!s || !kernel_ms || nsteps <= 0) return fail(CHEMO_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const bool grid = s->kp.has_grid && s->kp.chem_mode == 0;
    const bool overlap = grid && s->kp.overlap;
    const bool fused = grid && s->kp.fused_deposit;
    const bool variants = s->kp.hard_sphere || s->kp.kde;
    // in-cutoff pairs and candidate tests are counted into PROF_SLOTS
    // counters each (in the simulation's scratch) while profiling
    void *pcv = nullptr;
    if (int r = scratch(s, 2 * PROF_SLOTS * sizeof(unsigned long long), &pcv)) return r;
    unsigned long long *pc = static_cast<unsigned long long *>(pcv);
    CUDA_TRY(cudaMemsetAsync(pc, 0, 2 * PROF_SLOTS * sizeof(unsigned long long), st));
    // event pairs per step: particle, pde, scan, scatter, whole step
    std::vector<cudaEvent_t> ev((size_t)nsteps * 10, nullptr);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto &x : ev)
                if (x) cudaEventDestroy(x);
            return fail(CHEMO_ECUDA, "cudaEventCreate failed");
        }
    int r = CHEMO_OK;
    for (int64_t k = 0; k < nsteps && r == CHEMO_OK; ++k) {
        KP kp = view(s);
        kp.pair_count = pc;
        kp.test_count = pc + PROF_SLOTS;
        cudaEvent_t *e = &ev[(size_t)k * 10];
        cudaError_t err = cudaEventRecord(e[8], st);
        if (fused && !overlap) {
            if (err == cudaSuccess) err = cudaEventRecord(e[2], st);
            if (err == cudaSuccess) err = launch_pde(kp, s->cur, st, nullptr);
            if (err == cudaSuccess) err = cudaEventRecord(e[3], st);
        }
        if (overlap) {
            if (err == cudaSuccess) err = cudaEventRecord(s->ev_fork, st);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(s->aux, s->ev_fork, 0);
            if (err == cudaSuccess) err = cudaEventRecord(e[2], s->aux);
            if (err == cudaSuccess) err = launch_pde(kp, s->cur, s->aux, nullptr);
            if (err == cudaSuccess) err = cudaEventRecord(e[3], s->aux);
            if (err == cudaSuccess) err = cudaEventRecord(s->ev_join, s->aux);
        }
        // the particle kernels on the caller's stream, not on the step's
        // high-priority stream: with timing events between the kernels of
        // streams of different priority the profiled step came out 14 % slower
        // than the same step without them (which priorities make faster)
        if (err == cudaSuccess) err = cudaEventRecord(e[0], st);
        if (err == cudaSuccess) err = launch_step_particles(kp, s->cur, st, nullptr);
        if (err == cudaSuccess) err = cudaEventRecord(e[1], st);
        if (overlap && err == cudaSuccess) err = cudaStreamWaitEvent(st, s->ev_join, 0);
        if (err == cudaSuccess) err = cudaEventRecord(e[4], st);
        if (err == cudaSuccess && !variants) err = launch_scan(kp, st, nullptr);
        if (err == cudaSuccess) err = cudaEventRecord(e[5], st);
        if (err == cudaSuccess && !variants) err = launch_scatter(kp, s->cur, 1, st, nullptr);
        if (err == cudaSuccess && variants) {
            // the scan, scatter, correction and density kernels are timed
            // together in the scatter slot
            if (enqueue_sort_and_density(s, kp, st, nullptr) != CHEMO_OK) err = cudaErrorUnknown;
            s->cntp ^= 1;  // the sequence flipped the count buffers itself; undone by the flip below
        }
        if (err == cudaSuccess) err = cudaEventRecord(e[6], st);
        if (grid && !fused) {
            if (err == cudaSuccess) err = cudaEventRecord(e[2], st);
            if (err == cudaSuccess) err = launch_pde(kp, s->cur, st, nullptr);
            if (err == cudaSuccess) err = cudaEventRecord(e[3], st);
        }
        if (err == cudaSuccess) err = cudaEventRecord(e[9], st);
        if (err != cudaSuccess) r = fail(CHEMO_ECUDA, "profile: %s", cudaGetErrorString(err));
        if (grid) s->cur = fused ? (s->cur ^ 1) : (s->cur ^ (kp.pde_launches & 1));
        s->cntp ^= 1;
        s->step += 1;
    }
    if (r == CHEMO_OK) {
        cudaError_t err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) r = fail(CHEMO_ECUDA, "profile sync: %s", cudaGetErrorString(err));
    }
    if (r == CHEMO_OK) {
        double acc[5] = {0, 0, 0, 0, 0};
        const int pairs[5][2] = {{0, 1}, {2, 3}, {4, 5}, {5, 6}, {8, 9}};
        for (int64_t k = 0; k < nsteps; ++k) {
            cudaEvent_t *e = &ev[(size_t)k * 10];
            for (int q = 0; q < 5; ++q) {
                if (q == 1 && !grid) continue;
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, e[pairs[q][0]], e[pairs[q][1]]) == cudaSuccess) acc[q] += ms;
            }
        }
        for (int q = 0; q < 5; ++q) kernel_ms[q] = (float)(acc[q] / (double)nsteps);
        std::vector<unsigned long long> slots(2 * (size_t)PROF_SLOTS, 0ull);
        kernel_ms[5] = kernel_ms[6] = 0.f;
        if (cudaMemcpy(slots.data(), pc, slots.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) ==
            cudaSuccess) {
            unsigned long long cnt[2] = {0ull, 0ull};
            for (int k = 0; k < PROF_SLOTS; ++k) {
                cnt[0] += slots[(size_t)k];
                cnt[1] += slots[(size_t)PROF_SLOTS + k];
            }
            kernel_ms[5] = (float)((double)cnt[0] / (double)nsteps);
            kernel_ms[6] = (float)((double)cnt[1] / (double)nsteps);
        }
    }
    for (auto &x : ev) cudaEventDestroy(x);
    return r;
}

int chemo_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t n, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(CHEMO_EINVAL, "bad arguments");
    if (int r = check_mem_kind(mem_kind)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    if (mem_kind == CHEMO_MEM_DEVICE) {
        CUDA_TRY(launch_philox(seed, ctr, out, n, st));
        return CHEMO_OK;
    }
    const size_t bytes = (size_t)n * 16;
    const DevMem mem = eng_allocator();
    void *d = nullptr;
    size_t db = 0;
    if (int r = eng_mem_alloc(mem, &d, 2 * bytes + 32, &db)) return r;
    uint32_t *dc = (uint32_t *)d, *dout = (uint32_t *)((char *)d + bytes);
    cudaError_t e = cudaMemcpyAsync(dc, ctr, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_philox(seed, dc, dout, n, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, st);
    const cudaError_t es = cudaStreamSynchronize(st);  // the buffer is idle before it goes back
    if (e == cudaSuccess) e = es;
    eng_mem_release(mem, d, db);
    if (e != cudaSuccess) return fail(CHEMO_ECUDA, "philox: %s", cudaGetErrorString(e));
    return CHEMO_OK;
}

int chemo_init_positions(const chemo_params *params, int64_t n, int64_t n_alpha, float sigma_frac, float *pos_out,
                         uint8_t *species_out, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    ChemoRange nvtx_range("chemo_init_positions");
    if (!params) return fail(CHEMO_EINVAL, "params is required");
    if (int r = check_params(*params)) return r;
    if (n < 0 || n > (int64_t)ID_MASK + 1 || n_alpha < 0 || n_alpha > n)
        return fail(CHEMO_EINVAL, "need 0 <= n_alpha <= n <= 2^29");
    if (params->n_species < 2 && n_alpha < n) return fail(CHEMO_EINVAL, "beta cells need n_species >= 2");
    if (!(sigma_frac > 0.f) || !std::isfinite(sigma_frac)) return fail(CHEMO_EINVAL, "sigma_frac must be > 0");
    if (n > 0 && (!pos_out || !species_out)) return fail(CHEMO_EINVAL, "pos_out and species_out are required");
    if (int r = check_mem_kind(mem_kind)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    if (mem_kind == CHEMO_MEM_DEVICE) {
        CUDA_TRY(launch_init_positions(params->dim, params->boundary == 1, params->lo, params->hi, params->seed, n,
                                       n_alpha, sigma_frac, pos_out, species_out, st));
        return CHEMO_OK;
    }
    const size_t pb = (size_t)n * params->dim * sizeof(float);
    const DevMem mem = eng_allocator();
    void *d = nullptr;
    size_t db = 0;
    if (int r = eng_mem_alloc(mem, &d, pb + (size_t)n + 64, &db)) return r;
    float *dp = (float *)d;
    uint8_t *ds = (uint8_t *)d + ((pb + 15) & ~(size_t)15);
    cudaError_t e = launch_init_positions(params->dim, params->boundary == 1, params->lo, params->hi, params->seed, n,
                                          n_alpha, sigma_frac, dp, ds, st);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(pos_out, dp, pb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(species_out, ds, (size_t)n, cudaMemcpyDeviceToHost, st);
    const cudaError_t es = cudaStreamSynchronize(st);  // the buffer is idle before it goes back
    if (e == cudaSuccess) e = es;
    eng_mem_release(mem, d, db);
    if (e != cudaSuccess) return fail(CHEMO_ECUDA, "init_positions: %s", cudaGetErrorString(e));
    return CHEMO_OK;
}

// Stage entry points: results land in device scratch, then go to the caller.
static int stage_out(chemo_sim *s, void *dst, const void *src, size_t bytes, int mem_kind, cudaStream_t st)
{
    if (!dst || bytes == 0) return CHEMO_OK;
    CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                             mem_kind == CHEMO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    (void)s;
    return CHEMO_OK;
}

static int finish(chemo_sim *s, int mem_kind, void *stream)
{
    if (mem_kind == CHEMO_MEM_HOST) {
        CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
        return chemo_check(s, stream);
    }
    return CHEMO_OK;
}

int chemo_stall_scan(chemo_sim *s, uint32_t spin_limit, void *stream)
{
    g_last_error[0] = 0;
    if (!s || spin_limit == 0) return fail(CHEMO_EINVAL, "sim and a positive spin_limit are required");
    cudaStream_t st = (cudaStream_t)stream;
    KP k = view(s);
    if (scan_tiles(k) < 2) return fail(CHEMO_EINVAL, "the cell list has one scan tile: no tile waits on another");
    // The scan reads and clears the idle count buffer (all zero between
    // steps) and writes its offsets to scratch: the simulation's cell list
    // is left as it was.
    k.cnt_cur = k.cnt_nxt;
    void *tmp = nullptr;
    if (int r = scratch(s, ((size_t)k.ngroups + 1) * sizeof(uint32_t) + 256, &tmp)) return r;
    k.gstart = (uint32_t *)tmp;
    k.scan_spins = spin_limit;
    CUDA_TRY(launch_scan_from_tile(k, 1u, st));
    return CHEMO_OK;
}

int chemo_stage_bins(chemo_sim *s, int32_t *cells_out, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    if (s && s->kp.sub) return fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_stage_bins");
    if (!s || !cells_out) return fail(CHEMO_EINVAL, "sim and cells_out are required");
    if (int r = check_mem_kind(mem_kind)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)s->kp.n * s->kp.dim * sizeof(int32_t);
    void *tmp = nullptr;
    if (int r = scratch(s, bytes + 256, &tmp)) return r;
    CUDA_TRY(launch_stage_bins(view(s), (int32_t *)tmp, st));
    if (int r = stage_out(s, cells_out, tmp, bytes, mem_kind, st)) return r;
    return finish(s, mem_kind, stream);
}

int chemo_stage_sort(chemo_sim *s, uint32_t *ids_out, uint32_t *bin_start_out, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    if (s && s->kp.sub) return fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_stage_sort");
    if (!s) return fail(CHEMO_EINVAL, "sim is NULL");
    if (int r = check_mem_kind(mem_kind)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)s->kp.n * sizeof(uint32_t);
    void *tmp = nullptr;
    if (int r = scratch(s, bytes + 256, &tmp)) return r;
    if (ids_out) {
        CUDA_TRY(launch_stage_sort(view(s), (uint32_t *)tmp, nullptr, st));
        if (int r = stage_out(s, ids_out, tmp, bytes, mem_kind, st)) return r;
    }
    if (bin_start_out) {
        const size_t sb = ((size_t)s->kp.bin_slots + 1) * sizeof(uint32_t);
        void *t2;
        if (mem_kind == CHEMO_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(st));  // ids copied out before reuse
        if (int r = scratch(s, sb + 256, &t2)) return r;
        CUDA_TRY(launch_stage_sort(view(s), nullptr, (uint32_t *)t2, st));
        if (int r = stage_out(s, bin_start_out, t2, sb, mem_kind, st)) return r;
    }
    return finish(s, mem_kind, stream);
}

int chemo_stage_forces(chemo_sim *s, float *F_out, int32_t *count_out, uint64_t *idsum_out, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    if (s && s->kp.sub) return fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_stage_forces");
    if (!s || !F_out) return fail(CHEMO_EINVAL, "sim and F_out are required");
    if (int r = check_mem_kind(mem_kind)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = s->kp.n;
    const size_t fb = ((size_t)n * s->kp.dim * sizeof(float) + 255) & ~(size_t)255;
    const size_t cb = ((size_t)n * sizeof(int32_t) + 255) & ~(size_t)255;
    const size_t ib = (size_t)n * sizeof(uint64_t);
    void *tmp = nullptr;
    if (int r = scratch(s, fb + cb + ib + 256, &tmp)) return r;
    char *b = (char *)tmp;
    CUDA_TRY(launch_stage_forces(view(s), (float *)b, (int32_t *)(b + fb), (unsigned long long *)(b + fb + cb), st));
    if (int r = stage_out(s, F_out, b, (size_t)n * s->kp.dim * sizeof(float), mem_kind, st)) return r;
    if (int r = stage_out(s, count_out, b + fb, (size_t)n * sizeof(int32_t), mem_kind, st)) return r;
    if (int r = stage_out(s, idsum_out, b + fb + cb, ib, mem_kind, st)) return r;
    return finish(s, mem_kind, stream);
}

int chemo_stage_drift(chemo_sim *s, float *drift_out, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    if (s && s->kp.sub) return fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_stage_drift");
    if (!s || !drift_out) return fail(CHEMO_EINVAL, "sim and drift_out are required");
    if (int r = check_mem_kind(mem_kind)) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)s->kp.n * s->kp.dim * sizeof(float);
    void *tmp = nullptr;
    if (int r = scratch(s, bytes + 256, &tmp)) return r;
    CUDA_TRY(launch_stage_drift(view(s), s->cur, (float *)tmp, st));
    if (int r = stage_out(s, drift_out, tmp, bytes, mem_kind, st)) return r;
    return finish(s, mem_kind, stream);
}

int chemo_stage_deposit(chemo_sim *s, float *S_out, float *R_out, int mem_kind, void *stream)
{
    g_last_error[0] = 0;
    if (s && s->kp.sub) return fail(CHEMO_ENOTSUP, "%s: not for sub-domains", "chemo_stage_deposit");
    if (!s) return fail(CHEMO_EINVAL, "sim is NULL");
    if (int r = check_mem_kind(mem_kind)) return r;
    if (!s->kp.has_grid) return fail(CHEMO_EINVAL, "this simulation has no grid (chem_mode 1)");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t gb = ((size_t)s->kp.G * sizeof(float) + 255) & ~(size_t)255;
    void *tmp = nullptr;
    if (int r = scratch(s, 2 * gb, &tmp)) return r;
    float *dS = (float *)tmp, *dR = (float *)((char *)tmp + gb);
    CUDA_TRY(cudaMemsetAsync(tmp, 0, 2 * gb, st));
    if (s->kp.kde)
        CUDA_TRY(launch_kde(view(s), dS, dR, st, nullptr));
    else
        CUDA_TRY(launch_stage_deposit(view(s), dS, dR, st));
    if (int r = stage_out(s, S_out, dS, (size_t)s->kp.G * sizeof(float), mem_kind, st)) return r;
    if (int r = stage_out(s, R_out, dR, (size_t)s->kp.G * sizeof(float), mem_kind, st)) return r;
    return finish(s, mem_kind, stream);
}

}  // extern "C"
