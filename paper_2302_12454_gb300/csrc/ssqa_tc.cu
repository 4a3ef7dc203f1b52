// Host side of the persistent tensor-core path: feasibility check, shared
// memory plan, kernel parameters and launch (the kernel is in
// ssqa_tc_kernel.cuh).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <memory>
#include <new>
#include <vector>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <utility>

#include "ssqa_tc_kernel.cuh"

namespace ssqa {
namespace {
using namespace tc;

KernelFn pick(int d, bool both, bool track, bool bytes, bool f16, bool shfl) {
    if (shfl) switch (d) {
            case 0: return pick_shfl_d0(both, track, f16);
            case 1: return pick_shfl_d1(both, track, f16);
            case 2: return pick_shfl_d2(both, track, f16);
            default: return pick_shfl_d3(both, track, f16);
        }
    switch (d) {
        case 0: return pick_slot_d0(both, track, bytes, f16);
        case 1: return pick_slot_d1(both, track, bytes, f16);
        case 2: return pick_slot_d2(both, track, bytes, f16);
        default: return pick_slot_d3(both, track, bytes, f16);
    }
}

uint32_t half2_bits(float v) {
    const __half2 h = __floats2half2_rn(v, v);
    uint32_t u;
    std::memcpy(&u, &h, 4);
    return u;
}

// Every variant is configured once with the largest shared-memory carveout
// and opt-in size, so that launches for instances of different sizes (for
// example concurrent server requests) never need a different SM carveout.
void configure_once(KernelFn fn) {
    static std::mutex mu;
    static std::set<std::pair<int, KernelFn>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, fn})) return;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, int(cudaSharedmemCarveoutMaxShared));
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    done.insert({dev, fn});
}

struct Layout {
    int32_t W, WP, G, Tb;
    int32_t smem_A, smem_B, smem_slot, smem_h, smem_e, smem_bar, total;
};

bool plan(const TcImage &img, const AnnealArgs &a, Layout *L, std::string *why) {
    if (!img.ok) {
        *why = img.why;
        return false;
    }
    if (a.N != int32_t(img.h_unit.size())) {
        *why = "instance mismatch";
        return false;
    }
    if (a.R > kCT) {
        *why = "R > 128";
        return false;
    }
    if (img.nh > kMaxNh) {
        *why = "too many h digit columns";
        return false;
    }
    const int64_t jpmax = std::max<int64_t>(std::llabs(int64_t(a.jperp_min)),
                                            std::llabs(int64_t(a.jperp_min) + int64_t(a.jperp_step) * a.beta));
    const int64_t i0_top = a.i0_max > a.I0 ? a.i0_max : a.I0;
    if (i0_top + a.n_rnd + (a.both ? 2 : 1) * jpmax > 1024) {
        *why = "I0 + n_rnd + |J_perp| terms exceed the exact FP16 epilogue range (1024)";
        return false;
    }
    L->W = (a.N + 31) / 32;
    L->WP = L->W | 1;
    L->G = (a.N + 15) / 16;
    L->Tb = kCT / a.R;
    if (L->W > 4 * kMaxW) {  // each of the 4 warps of a column owns words part + 4 q, q < kMaxW
        *why = "N too large for the resident epilogue split";
        return false;
    }
    int32_t off = 0;
    L->smem_A = off;
    off += kCT * img.Kp;
    L->smem_B = off;
    off += img.Brows * img.Kp;
    L->smem_slot = off;
    off += (kCT * L->WP * 4 + 15) / 16 * 16;
    L->smem_h = off;  // h / jm: N floats, or N16 halves (zero beyond N)
    off += (std::max(a.N * 4, img.N16 * 2) + 15) / 16 * 16;
    L->smem_e = off;
    off += kCT * 8;
    L->smem_bar = off;
    off += 64 + 32 * 16;  // barriers, TMEM address, abort flag; the issuing warp's noise words
    L->total = off + 1024;  // alignment slack
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (optin <= 0) optin = 232448;
    if (L->total > optin) {
        *why = "operands do not fit in shared memory (" + std::to_string(L->total) + " bytes)";
        return false;
    }
    return true;
}

}  // namespace

bool tc_supported(const TcImage &img, const AnnealArgs &a, std::string *why) {
    Layout L;
    return plan(img, a, &L, why);
}

TcVariant tc_variant(const TcImage &img, const AnnealArgs &a) {
    // byte counters: counters fit a biased byte, alpha = 1, and a fresh start
    // (resumed counters may lie outside the byte range); shuffle exchange
    // when R divides 32; FP16 accumulator when every partial sum is an
    // integer of magnitude <= 2048, and so is D + h / jm (the energy's term)
    TcVariant v;
    const int32_t i0_top = a.i0_max > a.I0 ? a.i0_max : a.I0;
    v.bytes = i0_top <= 127 && a.alpha == 1 && a.init_mode != SSQA_INIT_FROM_STATE;
    v.shfl = v.bytes && 32 % a.R == 0;
    v.f16 = v.bytes && img.max_row_sum + img.max_h_unit <= 2048;
    return v;
}

// Kernel parameters, shared-memory layout and variant of one problem (no
// device work); SSQA_ERR_UNSUPPORTED when the resident kernel cannot take it.
static int build_params(const TcImage &img, const DeviceCopy &dc, const AnnealArgs &a, TcParams *pp, Layout *Lp,
                        TcVariant *vp) {
    Layout &L = *Lp;
    std::string why;
    if (!plan(img, a, &L, &why)) return fail(SSQA_ERR_UNSUPPORTED, "tensor path: " + why);
    TcParams &p = *pp;
    std::memset(&p, 0, sizeof(p));
    p.a = a;
    p.b_img = dc.tc_b;
    p.h_unit = dc.tc_h_unit;
    p.Kp = img.Kp;
    p.N16 = img.N16;
    p.nh = img.nh;
    p.nchunk = img.nchunk;
    p.Brows = img.Brows;
    p.jm = img.jm;
    p.Tb = L.Tb;
    p.W = L.W;
    p.WP = L.WP;
    p.G = L.G;
    p.crow[0] = img.chunk_rows[0];
    p.crow[1] = img.chunk_rows[1];
    const TcVariant var = tc_variant(img, a);
    *vp = var;
    const bool fast = var.bytes, f16 = var.f16;
    for (int ch = 0; ch < 2; ++ch) {
        // instruction descriptor, kind::f8f6f4: D f16 (bits 4-5 = 0) or f32 (1),
        // A and B E4M3 (format 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
        p.idesc[ch] = ((f16 ? 0u : 1u) << 4) | (uint32_t(img.chunk_rows[ch] >> 3) << 17) | (uint32_t(kCT >> 4) << 24);
    }
    uint32_t tc = 32;
    while (tc < uint32_t(img.Brows)) tc <<= 1;
    p.tmem_cols = tc;
    for (int m = 0; m < img.nh; ++m) p.a_w[m] = img.a_w[m];
    p.JM2 = half2_bits(float(img.jm));
    p.NR2 = half2_bits(float(a.n_rnd));
    p.bias = fast ? 1152.f : 0.f;
    p.i0_levels = 1;
    p.i0_mult = 2;
    p.i0_tau = 1 << 30;
    if (a.i0_max > a.I0) {
        for (int64_t v = a.I0; v < a.i0_max; v *= a.i0_mult) ++p.i0_levels;
        p.i0_mult = a.i0_mult;
        p.i0_tau = a.i0_tau;
    }
    p.smem_A = L.smem_A;
    p.smem_B = L.smem_B;
    p.smem_slot = L.smem_slot;
    p.smem_h = L.smem_h;
    p.smem_e = L.smem_e;
    p.smem_bar = L.smem_bar;
    p.wait_clocks = wait_limit_clocks();
    return SSQA_OK;
}

int tc_anneal(const TcImage &img, const DeviceCopy &dc, const AnnealArgs &a, void *stream) {
    Layout L;
    TcParams p;
    TcVariant var;
    if (int rc = build_params(img, dc, a, &p, &L, &var)) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *err = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&err), sizeof(int), st);
    if (e) return fail(SSQA_ERR_OOM, std::string("tensor path: ") + cudaGetErrorString(e));
    cudaMemsetAsync(err, 0, sizeof(int), st);
    p.err = err;
    KernelFn fn = pick(a.delay, a.both != 0, a.track_best, var.bytes, var.f16, var.shfl);
    configure_once(fn);
    const int64_t grid = (int64_t(a.trials) + L.Tb - 1) / L.Tb;
    fn<<<unsigned(grid), kThreads, L.total, st>>>(p);
    e = cudaGetLastError();
    int herr = 0;
    if (!e) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    cudaFreeAsync(err, st);
    if (e) return fail(SSQA_ERR_DEVICE, std::string("tensor path kernel: ") + cudaGetErrorString(e));
    if (herr) return fail(SSQA_ERR_TIMEOUT, "tensor path: a bounded wait for the tensor cores timed out");
    return SSQA_OK;
}

int tc_batch_key(const TcImage &img, const AnnealArgs &a) {
    Layout L;
    std::string why;
    if (!plan(img, a, &L, &why)) return -1;
    const TcVariant v = tc_variant(img, a);
    if (!tc::pick_batch(a.delay, a.both != 0, a.track_best, v.bytes, v.f16, v.shfl)) return -1;
    return (a.both ? 4 : 0) | (a.track_best ? 2 : 0) | (v.f16 ? 1 : 0);
}

int tc_anneal_batch(const TcBatchItem *items, int count, int *launches, void *stream) {
    using namespace tc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<TcParams> ps(count);
    std::vector<Layout> Ls(count);
    std::vector<BatchFn> fns(count);
    std::vector<std::pair<BatchFn, int>> order;  // batchable items grouped by kernel variant
    for (int i = 0; i < count; ++i) {
        TcVariant var;
        if (int rc = build_params(*items[i].img, *items[i].dc, items[i].a, &ps[i], &Ls[i], &var)) return rc;
        const AnnealArgs &a = items[i].a;
        fns[i] = pick_batch(a.delay, a.both != 0, a.track_best, var.bytes, var.f16, var.shfl);
        if (fns[i]) order.emplace_back(fns[i], i);
    }
    // variants without a batched kernel run alone
    for (int i = 0; i < count; ++i)
        if (!fns[i]) {
            if (int rc = tc_anneal(*items[i].img, *items[i].dc, items[i].a, stream)) return rc;
            if (launches) ++*launches;
        }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<BatchFn, int> &x, const std::pair<BatchFn, int> &y) {
                         return reinterpret_cast<uintptr_t>(x.first) < reinterpret_cast<uintptr_t>(y.first);
                     });
    int *err = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&err), sizeof(int), st);
    if (e) return fail(SSQA_ERR_OOM, std::string("tensor path: ") + cudaGetErrorString(e));
    cudaMemsetAsync(err, 0, sizeof(int), st);
    std::unique_ptr<TcBatch> b(new (std::nothrow) TcBatch());
    if (!b) {
        cudaFreeAsync(err, st);
        return fail(SSQA_ERR_OOM, "tensor path: out of host memory");
    }
    size_t k = 0;
    while (!e && k < order.size()) {
        // one launch: consecutive items of one variant, at most kMaxBatch
        const BatchFn fn = order[k].first;
        std::memset(b.get(), 0, sizeof(TcBatch));
        int smem = 0;
        int64_t ctas = 0;
        while (k < order.size() && order[k].first == fn && b->count < kMaxBatch) {
            const int i = order[k].second;
            TcParams &p = ps[i];
            p.err = err;
            const int64_t grid = (int64_t(items[i].a.trials) + Ls[i].Tb - 1) / Ls[i].Tb;
            b->first[b->count] = int32_t(ctas);
            b->items[b->count] = p;
            ++b->count;
            ctas += grid;
            smem = std::max(smem, Ls[i].total);
            ++k;
        }
        b->first[b->count] = int32_t(ctas);
        configure_once(reinterpret_cast<KernelFn>(fn));
        fn<<<unsigned(ctas), kThreads, smem, st>>>(*b);
        e = cudaGetLastError();
        if (!e && launches) ++*launches;
    }
    int herr = 0;
    if (!e) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    cudaFreeAsync(err, st);
    if (e) return fail(SSQA_ERR_DEVICE, std::string("batched tensor path kernel: ") + cudaGetErrorString(e));
    if (herr) return fail(SSQA_ERR_TIMEOUT, "batched tensor path: a bounded wait for the tensor cores timed out");
    return SSQA_OK;
}

}  // namespace ssqa
