// ssqa_anneal_noalloc: the plain CUDA-core anneal (one launch per cycle) for
// callers that cannot allocate device memory.
//
// Who cannot allocate: plugins inside host frameworks that hand out all
// device memory from their own pools and forbid cudaMalloc after start-up,
// real-time loops in which an allocation (which may synchronise the device)
// would break the timing, and deployments that fix their whole device
// footprint at initialisation.
// Such callers pass every input and output buffer themselves; the scratch
// this path needs between cycle launches (the spin history ring and two
// per-column energy accumulators) lives in one file-scope device array that
// the library holds on every GPU that loads it, until the process exits.
//
// The paper has no counterpart: this is an allocation-free way to call the
// same computation as ssqa_anneal with SSQA_ALGO_PLAIN.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ssqa_internal.h"

namespace {

// Fixed scratch: 16 MiB.  The plain path needs (delay + 2) * trials * R *
// roundup(N, 16) bytes of spin history plus 16 bytes per column (plus
// alignment); larger problems are rejected.
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device; the name alone is a host-side stand-in, not a device address).
int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ssqa::fail(SSQA_ERR_DEVICE, std::string("ssqa_anneal_noalloc: no CUDA device: ") + cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= kMaxDevices) return ssqa::fail(SSQA_ERR_DEVICE, "ssqa_anneal_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return ssqa::fail(SSQA_ERR_DEVICE,
                              std::string("ssqa_anneal_noalloc: scratch address lookup failed: ") + cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SSQA_OK;
}

int check_params(int32_t N, const ssqa_params *p, const ssqa_result *r) {
    using ssqa::fail;
    if (N < 1 || N > 65536) return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: N must be in 1..65536");
    if (p->R < 1 || p->R > 128 || p->trials < 1 || p->cycles < 0)
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: R in 1..128, trials >= 1, cycles >= 0");
    if (p->I0 < 1 || p->I0 > 16383 || p->alpha < 1 || p->alpha > 2 * p->I0 || p->n_rnd < 0 || p->n_rnd > (1 << 20))
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: I0, alpha or n_rnd out of range");
    if (p->i0_max > p->I0) {
        int64_t v = p->I0;
        while (p->i0_mult >= 2 && v < p->i0_max) v *= p->i0_mult;
        if (p->i0_mult < 2 || p->i0_tau < 1 || v != p->i0_max || p->i0_max > 16383)
            return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: bad I0 schedule");
    }
    if (p->beta < 1 || p->tau < 1 || (int64_t(p->jperp_max) - p->jperp_min) % p->beta ||
        p->jperp_min < -(1 << 20) || p->jperp_min > (1 << 20) || p->jperp_max < -(1 << 20) || p->jperp_max > (1 << 20))
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: bad J_perp schedule");
    if (p->delay < 0 || p->delay > 3 || (p->coupling != SSQA_COUPLING_UPPER && p->coupling != SSQA_COUPLING_BOTH) ||
        p->init_mode < 0 || p->init_mode > 2)
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: bad delay, coupling or init mode");
    if (p->start_cycle < 0 || int64_t(p->start_cycle) + p->cycles > 0xFFFFFFFEll ||
        int64_t(p->trial_offset) + p->trials > 0xFFFFFFFFll)
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: cycle or trial range out of 32 bits");
    if (!(p->flags & SSQA_FLAG_DEVICE_PTRS) || (p->flags & ~(SSQA_FLAG_DEVICE_PTRS | SSQA_FLAG_TRACK_BEST)))
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: flags must include SSQA_FLAG_DEVICE_PTRS");
    if (!r->sigma || !r->is_state) return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: sigma and is_state required");
    if (p->init_mode == SSQA_INIT_FROM_STATE && p->delay > 0 && !r->sigma_hist)
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: resuming with delay > 0 needs sigma_hist");
    if ((p->flags & SSQA_FLAG_TRACK_BEST) && (!r->e_best || !r->best_cycle))
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: TRACK_BEST needs e_best and best_cycle");
    if (r->e_trace && !(p->flags & SSQA_FLAG_TRACK_BEST))
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: e_trace needs SSQA_FLAG_TRACK_BEST");
    return SSQA_OK;
}

// The kernels read J rows as 16-byte vectors, h and the counters as int32,
// and write the energies as int64: a caller's pointer that is not aligned to
// its access width (an offset view of a larger buffer, say) is rejected here,
// before anything is launched, instead of faulting on the device.
int check_alignment(const int8_t *J_padded, const int32_t *h, const ssqa_result *r) {
    auto bad = [](const void *q, uintptr_t a) { return q != nullptr && (reinterpret_cast<uintptr_t>(q) % a) != 0; };
    if (bad(J_padded, 16)) return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: J_padded must be 16-byte aligned");
    if (bad(h, 4) || bad(r->is_state, 4) || bad(r->best_cycle, 4))
        return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: h, is_state and best_cycle must be 4-byte aligned");
    if (bad(r->e_final, 8) || bad(r->e_best, 8) || bad(r->e_trace, 8))
        return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: e_final, e_best and e_trace must be 8-byte aligned");
    return SSQA_OK;
}

}  // namespace

extern "C" int ssqa_anneal_noalloc(int32_t N, const int8_t *J_padded, const int32_t *h, const ssqa_params *params,
                                   ssqa_result *out, void *cuda_stream) {
    if (!J_padded || !h || !params || !out) return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_noalloc: NULL argument");
    if (int rc = check_params(N, params, out)) return rc;
    if (int rc = check_alignment(J_padded, h, out)) return rc;
    const ssqa_params &p = *params;
    ssqa::AnnealArgs a{};
    a.N = N;
    a.R = p.R;
    a.trials = p.trials;
    a.cycles = p.cycles;
    a.I0 = p.I0;
    a.alpha = p.alpha;
    a.n_rnd = p.n_rnd;
    a.jperp_min = p.jperp_min;
    a.jperp_step = (p.jperp_max - p.jperp_min) / p.beta;
    a.beta = p.beta;
    a.tau = p.tau;
    a.delay = p.delay;
    a.both = p.coupling == SSQA_COUPLING_BOTH;
    a.init_mode = p.init_mode;
    a.start_cycle = p.start_cycle;
    a.trial_offset = p.trial_offset;
    a.seed = p.seed;
    a.i0_max = p.i0_max;
    a.i0_mult = p.i0_mult;
    a.i0_tau = p.i0_tau;
    a.track_best = (p.flags & SSQA_FLAG_TRACK_BEST) != 0;
    a.J = J_padded;
    a.J_pad = J_padded;
    a.Np = (N + 15) / 16 * 16;
    a.h = h;
    a.sigma = out->sigma;
    a.hist = p.delay ? out->sigma_hist : nullptr;
    a.Is = out->is_state;
    a.e_final = out->e_final;
    a.e_best = a.track_best ? out->e_best : nullptr;
    a.best_cycle = a.track_best ? out->best_cycle : nullptr;
    a.e_trace = a.track_best ? out->e_trace : nullptr;
    const size_t need = ssqa::plain_scratch_bytes(a);
    if (need > kNoallocScratchBytes)
        return ssqa::fail(SSQA_ERR_INVALID_ARG,
                          "ssqa_anneal_noalloc: problem needs " + std::to_string(need) + " bytes of scratch, more than the fixed " +
                              std::to_string(kNoallocScratchBytes) + " (reduce trials, R or N, or use ssqa_anneal)");
    void *scratch = nullptr;
    if (int rc = scratch_address(&scratch)) return rc;
    return ssqa::plain_anneal(a, scratch, cuda_stream);
}
