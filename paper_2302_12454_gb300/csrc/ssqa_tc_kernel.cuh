// Persistent tensor-core kernel of SSQA for sm_103a (tcgen05 + TMEM).
//
// One CTA owns 128 spin columns c = (trial, replica k) -- whole trials, so
// the replica ring of Eq. 4 / Fig. 2 stays inside the CTA -- and runs every
// annealing cycle of Eq. 6a-6c for them in one launch, with no global-memory
// traffic inside the cycle loop:
//
//   shared memory  A = sigma(t) as FP8 E4M3 (+1/-1), 128 x Kp, rewritten each
//                  cycle by the epilogue; B = J / jm and the h digits, read
//                  once from global memory; h / jm for the energy; with the
//                  shared-memory exchange, one word-per-32-spins bit slot
//                  with sigma(t - d) of every column for the replica term.
//   tensor memory  D[c][i] = sum_j sigma_{j,c}(t) J_ij / jm + h_i / jm, FP32
//                  or FP16, produced by tcgen05.mma kind::f8f6f4 in two
//                  N-chunks of rows (exact: every operand is a small integer
//                  and every partial sum is below 2^14; FP16 only where every
//                  partial sum, and D + h / jm, is at most 2048).
//   registers      the integral counters Is (Eq. 6b) as biased bytes or
//                  packed half2, and the thread's own spin history as bit
//                  words.
//
// Warp roles: all 16 warps run the epilogue (warp w reads TMEM lanes
// 32*(w%4).., i.e. columns, and a quarter (w/4) of the spins); warp 15 also
// allocates TMEM and its lane 0 issues the MMAs.  Per cycle:
//   MMA(sigma(t)) -> commit per chunk -> epilogue: D -> local field (Eq. 6a)
//   -> counter (Eq. 6b) -> sign (Eq. 6c) -> sigma(t+1) into A -> barrier;
// the first chunk's epilogue runs while the second chunk's MMAs do.  The
// cycle loop is kept small (the final energy of untracked runs is a separate
// pass after it): at 16 warps x 128 registers its speed follows its code size.
// Epilogue arithmetic is exact in FP16: the local field is an integer, and
// any value above 2048 in magnitude (the only ones FP16 rounds) saturates
// the counter in the same direction as the exact value, because the host
// limits I0 + n_rnd + |J_perp| terms to 1024.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstring>

#include "philox.cuh"
#include "ssqa_internal.h"

namespace ssqa {
namespace tc {

constexpr int kCT = 128;                 // spin columns per CTA (MMA M)
constexpr int kEpiWarps = 16;
constexpr int kThreads = kEpiWarps * 32;
constexpr int kMaxG = 8;                 // 16-spin granules per epilogue thread
constexpr int kMaxW = 4;                 // 32-spin words per epilogue thread
constexpr uint32_t kSignPair = 0x80008000u;
constexpr int kMaxNh = 16;
// Waits for the kernel's own operations in flight (MMAs, copies) before it
// exits after an abort: always this bound, whatever the caller's limit.
constexpr long long kDrainCycles = 4000000000LL;

struct TcParams {
    AnnealArgs a;
    const uint8_t *b_img;
    const int32_t *h_unit;
    int32_t Kp, N16, nh, nchunk, Brows, jm, Tb, W, WP, G;
    int32_t crow[2];
    uint32_t idesc[2];
    uint32_t tmem_cols;
    uint8_t a_w[kMaxNh];
    uint32_t JM2, NR2;
    float bias;                // counter offset of the FP16 epilogue
    int32_t i0_levels, i0_mult, i0_tau;  // I0 schedule (1 level: fixed I0)
    int32_t smem_A, smem_B, smem_slot, smem_h, smem_e, smem_bar;
    long long wait_clocks;     // bound of every wait for the tensor cores (SM clocks)
    int *err;
};

// ----------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Limits below this many clocks are honoured by polling without suspending.
constexpr long long kPollBelow = 1LL << 20;
// Wait for phase `parity` of an mbarrier; false after `limit` SM clocks.  The
// bound uses the SM clock counter: reading it costs no more than an ALU op,
// where a global-timer read on every poll slowed pipelines that wait once per
// stage.  try_wait may suspend the thread until the phase completes (for a
// hardware-defined time), which would overrun a short limit: those poll with
// test_wait instead.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    if (limit < kPollBelow) {
        const long long t0 = clock64();
        while (!mbar_test_wait(bar, parity))
            if (clock64() - t0 > limit) return false;
        return true;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D(tmem) (+)= A(smem) * B(smem)^T, FP8 operands, FP32 accumulate.
__device__ __forceinline__ void mma_f8f6f4(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// acc + lo + hi of an FP16 pair, each half converted exactly to FP32.
__device__ __forceinline__ float add_h2_to_f32(float acc, uint32_t h2) {
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %1;\n\t"
        "add.rn.f32.f16 %0, lo, %0;\n\tadd.rn.f32.f16 %0, hi, %0;\n\t}"
        : "+f"(acc)
        : "r"(h2));
    return acc;
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 lanes x 16 consecutive 32-bit TMEM columns, issued without waiting;
// the registers are valid only after tmem_ld_wait on the same array.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
// Wait for every outstanding tcgen05.ld of this thread; `r` is tied to the
// wait so that no use of it is scheduled before the data has arrived.
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])::"memory");
}
// 32 lanes x 16 consecutive 16-bit TMEM columns (an FP16 accumulator), packed
// two per register (column 2i in the low half), issued without waiting.
__device__ __forceinline__ void tmem_ld16h_issue(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.pack::16b.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_wait8(uint32_t (&r)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])::"memory");
}
// Shared-memory matrix descriptor (tcgen05), no swizzle, K-major:
// core matrices of 8 rows x 16 bytes; LBO = stride between K-adjacent core
// matrices, SBO = stride between 8-row groups; version field = 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t((lbo & 0x3FFFFu) >> 4) << 16) |
           (uint64_t((sbo & 0x3FFFFu) >> 4) << 32) | (uint64_t(1) << 46);
}

// ------------------------------------------------------------- half2 helpers
__device__ __forceinline__ uint32_t h2u(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}
__device__ __forceinline__ __half2 u2h(uint32_t u) {
    __half2 h;
    memcpy(&h, &u, 4);
    return h;
}
// FP32 pair (lo, hi) -> packed half2 (round to nearest; exact for |x| <= 2048)
__device__ __forceinline__ uint32_t pack_h2(uint32_t lo_bits, uint32_t hi_bits) {
    return h2u(__floats2half2_rn(__uint_as_float(lo_bits), __uint_as_float(hi_bits)));
}
// Element offset of (row r, k) in the core-matrix layout.
__device__ __forceinline__ uint32_t cm_off(int r, int k, int Kp) {
    return uint32_t((r >> 3) * (Kp * 8) + (k >> 4) * 128 + (r & 7) * 16 + (k & 15));
}
// Four sign-carrying half2 words (bits 15/31) -> 16 FP8 E4M3 bytes +1/-1.
__device__ __forceinline__ uint4 fp8_bytes(const uint32_t (&s)[8]) {
    uint4 o;
    o.x = (__byte_perm(s[0], s[1], 0x7531) & 0x80808080u) | 0x38383838u;
    o.y = (__byte_perm(s[2], s[3], 0x7531) & 0x80808080u) | 0x38383838u;
    o.z = (__byte_perm(s[4], s[5], 0x7531) & 0x80808080u) | 0x38383838u;
    o.w = (__byte_perm(s[6], s[7], 0x7531) & 0x80808080u) | 0x38383838u;
    return o;
}

// Keep only the bytes of spins < N in a 16-byte granule starting at spin i0.
__device__ __forceinline__ uint4 mask_tail(uint4 b, int i0, int N) {
    auto m = [&](int q) -> uint32_t {
        const int nv = N - (i0 + 4 * q);
        return nv >= 4 ? 0xFFFFFFFFu : (nv <= 0 ? 0u : ((1u << (8 * nv)) - 1u));
    };
    b.x &= m(0);
    b.y &= m(1);
    b.z &= m(2);
    b.w &= m(3);
    return b;
}

// Sign bit (set = -1) of spin i inside a 32-spin word with the pair layout.
__device__ __forceinline__ uint32_t word_bit(uint32_t w, uint32_t i) { return (w >> spin_bit_pos(i)) & 1u; }

// ------------------------------------------------------------------- kernel
// kFast (byte counters): I0 <= 127 (each counter Is kept as the byte Is + 128,
// four per register) and alpha = 1 (the counter update is a clamp).  Otherwise
// the counters are half2 and Eq. 6b is applied with a compare.  In both,
// counters are handled in FP16 with an offset `bias` (1152 for byte counters,
// where half(1024 + b) holds the byte b exactly, 0 otherwise).
// kShfl (byte counters and R dividing 32): ring neighbours are lanes of the
// same warp and the spin history is exchanged by shuffles; otherwise through a
// shared-memory slot, with a barrier before it is rewritten.
// kF16 (byte counters only): the accumulator is FP16 (every partial sum is an
// integer of magnitude <= 2048, exact in FP16), read from TMEM as packed half2
// pairs, so the epilogue needs no FP32 -> FP16 conversion.
// One CTA's whole anneal: column group `cta` of the problem described by p.
template <int D, bool kBoth, bool kTrack, bool kFast, bool kF16, bool kShfl>
__device__ __forceinline__ void cta_anneal(const TcParams &p, const int cta) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = sm + p.smem_A;
    uint8_t *sB = sm + p.smem_B;
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + p.smem_slot);
    float *sh = reinterpret_cast<float *>(sm + p.smem_h);
    unsigned long long *eacc = reinterpret_cast<unsigned long long *>(sm + p.smem_e);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + p.smem_bar);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 3);
    uint64_t *drain = bars + 4;                        // completion of every MMA issued, before exit
    uint4 *xph = reinterpret_cast<uint4 *>(bars + 8);  // [32] noise words of the issuing warp's lanes

    const AnnealArgs &a = p.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // The last warp allocates TMEM and (lane 0) issues the MMAs.  Issue blocks
    // while the tensor cores work, so the issuing warp starts its epilogue late:
    // it is the warp of the last part, which owns the fewest spin words.
    const bool mma_warp = warp == kEpiWarps - 1;
    const int Kp = p.Kp;
    const int64_t trial0 = int64_t(cta) * p.Tb;
    const int ntr = int(a.trials - trial0 < p.Tb ? a.trials - trial0 : p.Tb);
    const int vcols = ntr * a.R;
    const int64_t col0 = trial0 * a.R;  // global column of local column 0
    const bool need_final = a.e_final != nullptr || kTrack;
    // Tracking variants compute E every cycle, the final one in one more loop
    // iteration; the others take E(sigma(t0 + cycles)) in a separate pass
    // after the loop, which keeps the energy code out of the cycle loop.
    const int iters = a.cycles + (kTrack ? 1 : 0);

    // ---------------------------------------------------------------- set-up
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (mma_warp) {
        tmem_alloc(tmem_holder, p.tmem_cols);
        tmem_relinquish();
    }
    {
        uint4 *A4 = reinterpret_cast<uint4 *>(sA);
        for (int x = tid; x < kCT * Kp / 16; x += kThreads) A4[x] = make_uint4(0, 0, 0, 0);
        const uint4 *g4 = reinterpret_cast<const uint4 *>(p.b_img);
        uint4 *B4 = reinterpret_cast<uint4 *>(sB);
        for (int x = tid; x < p.Brows * Kp / 16; x += kThreads) B4[x] = __ldg(&g4[x]);
        if constexpr (kF16) {
            __half *shh = reinterpret_cast<__half *>(sh);
            for (int x = tid; x < p.N16; x += kThreads)
                shh[x] = __float2half_rn(x < a.N ? float(__ldg(&p.h_unit[x])) : 0.f);
        } else {
            for (int x = tid; x < a.N; x += kThreads) sh[x] = float(__ldg(&p.h_unit[x]));
        }
        for (int x = tid; x < kCT; x += kThreads) eacc[x] = 0ull;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    for (int x = tid; x < vcols * p.nh; x += kThreads) {
        const int c = x / p.nh, m = x % p.nh;
        sA[cm_off(c, p.N16 + m, Kp)] = p.a_w[m];
    }
    const uint32_t tmem = *tmem_holder;

    // epilogue thread identity
    const int qd = warp & 3, part = warp >> 2;
    const int c = qd * 32 + lane;                      // local column = TMEM lane
    const bool valid = c < vcols;
    const int lt = valid ? c / a.R : 0, k = valid ? c % a.R : 0;
    const uint32_t trial_g = a.trial_offset + uint32_t(trial0 + lt);
    const int nb_up = lt * a.R + (k + 1) % a.R;
    const int nb_dn = lt * a.R + (k + a.R - 1) % a.R;
    // with R dividing 32 a trial never straddles a warp: neighbours are lanes
    const int src_up = nb_up & 31, src_dn = nb_dn & 31;
    // spin words owned by this thread: part + 4 q, q = 0..3 (one Philox call,
    // counter `part`, gives all four noise words; every part has granules in
    // the first MMA chunk).  Granule g = 2 q + h covers spins 16 (2 (part +
    // 4 q) + h) .. +15 and exists when that start is below N.
    auto gran_of = [&](int g) { return 2 * (part + 4 * (g >> 1)) + (g & 1); };
    const uint32_t key0 = uint32_t(a.seed), key1 = uint32_t(a.seed >> 32);
    const uint32_t taddr_lane = tmem + (uint32_t(qd * 32) << 16);

    // counters: fast variant 4 biased bytes per word, general half2 pairs
    uint32_t IsR[kMaxG][kFast ? 4 : 8];
    uint32_t H[D + 1][kMaxW];  // own spin history, H[l] = sigma(t - l), bit words
#pragma unroll
    for (int g = 0; g < kMaxG; ++g)
#pragma unroll
        for (int q = 0; q < (kFast ? 4 : 8); ++q) IsR[g][q] = kFast ? 0x80808080u : 0u;
#pragma unroll
    for (int l = 0; l <= D; ++l)
#pragma unroll
        for (int q = 0; q < kMaxW; ++q) H[l][q] = 0u;
    int64_t e_best = LLONG_MAX;
    int32_t best_cycle = -1;
    int64_t e_fin = 0;

    // --------------------------------------------- initial state sigma(t0)
    if (valid) {
        const int64_t gcol = col0 + c;
        const int64_t ht = trial0 + lt;
#pragma unroll
        for (int g = 0; g < kMaxG; ++g) {
            const int gg = gran_of(g);
            if (gg >= p.G) continue;
            const int i0 = gg * 16;
            const int half = g & 1;
            const int lw = g >> 1;
            uint32_t s[8];
            if (a.init_mode == SSQA_INIT_FROM_STATE) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i = i0 + 2 * q;
                    const uint32_t lo = (i < a.N && a.sigma[gcol * a.N + i] < 0) ? 0x8000u : 0u;
                    const uint32_t hi = (i + 1 < a.N && a.sigma[gcol * a.N + i + 1] < 0) ? 0x80000000u : 0u;
                    s[q] = lo | hi;
                    if (!kFast) {
                        const int32_t v0 = i < a.N ? a.Is[gcol * a.N + i] : 0;
                        const int32_t v1 = i + 1 < a.N ? a.Is[gcol * a.N + i + 1] : 0;
                        IsR[g][q] = h2u(__floats2half2_rn(float(v0), float(v1)));
                    }
                }
            } else {
                uint32_t w = 0xFFFFFFFFu;  // all -1
                if (a.init_mode == SSQA_INIT_RANDOM)
                    w = noise_word(a.seed, uint32_t(i0), uint32_t(k), trial_g, 0xFFFFFFFFu);
#pragma unroll
                for (int q = 0; q < 8; ++q) s[q] = (w << (half * 8 + q)) & kSignPair;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) H[0][lw] |= s[q] >> (half * 8 + q);
            uint4 b = fp8_bytes(s);
            if (i0 + 16 > a.N) b = mask_tail(b, i0, a.N);  // spins beyond N stay 0 in A
            *reinterpret_cast<uint4 *>(sA + cm_off(c, i0, Kp)) = b;
        }
        // older levels sigma(t0 - l)
#pragma unroll
        for (int l = 1; l <= D; ++l) {
#pragma unroll
            for (int q = 0; q < kMaxW; ++q) {
                if (gran_of(2 * q) >= p.G) continue;
                if (a.init_mode == SSQA_INIT_FROM_STATE) {
                    uint32_t w = 0;
                    for (int e = 0; e < 32; ++e) {
                        const int i = (part + 4 * q) * 32 + e;
                        if (i < a.N && a.hist[((ht * D + (l - 1)) * a.R + k) * int64_t(a.N) + i] < 0)
                            w |= 1u << spin_bit_pos(uint32_t(i));
                    }
                    H[l][q] = w;
                } else {
                    H[l][q] = H[0][q];
                }
            }
        }
        if (!kShfl)
#pragma unroll
            for (int q = 0; q < kMaxW; ++q)
                if (gran_of(2 * q) < p.G) slot[c * p.WP + part + 4 * q] = H[D][q];
    }
    fence_proxy_async();
    tc_fence_before();
    bar_sync(1, kThreads);

    // MMA descriptors: advancing one K-step (32 bytes of each row pair of
    // core matrices = 256 bytes) adds 16 to the start-address field
    uint64_t adesc0 = 0, bdesc0[2] = {0, 0};
    if (mma_warp && lane == 0) {
        adesc0 = smem_desc(smem_u32(sA), 128u, uint32_t(Kp) * 8u);
        bdesc0[0] = smem_desc(smem_u32(sB), 128u, uint32_t(Kp) * 8u);
        bdesc0[1] = smem_desc(smem_u32(sB) + uint32_t(p.crow[0] / 8) * uint32_t(Kp) * 8u, 128u, uint32_t(Kp) * 8u);
    }
    const int ksteps = Kp / 32;
    // E' = -(jm/2) sum_i sigma_i (D_i + h_i/jm) of one granule (spins i0 ..
    // i0 + 15, half `half` of the bit word sw = sigma), added to es
    auto energy_add = [&](const uint32_t (&f)[kF16 ? 8 : 16], const uint32_t sw, const int half, const int i0,
                          float es) -> float {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = half * 8 + q;
            const int i = i0 + 2 * q;
            if constexpr (kF16) {
                // D + h/jm as an FP16 pair (exact: |D_i| + |h_i/jm| <= 2048 on this
                // variant; zero beyond N), sign-flipped by sigma, added into FP32
                const uint32_t hp = reinterpret_cast<const uint32_t *>(sh)[i >> 1];
                const uint32_t y2 = h2u(__hadd2(u2h(f[q]), u2h(hp))) ^ ((sw << j) & kSignPair);
                es = add_h2_to_f32(es, y2);
            } else {
                const float y0 = __uint_as_float(f[2 * q]) + (i < a.N ? sh[i] : 0.f);
                const float y1 = __uint_as_float(f[2 * q + 1]) + (i + 1 < a.N ? sh[i + 1] : 0.f);
                const uint32_t sl = (sw << (16 + j)) & 0x80000000u;
                const uint32_t shi = (sw << j) & 0x80000000u;
                es += __uint_as_float(__float_as_uint(y0) ^ sl);
                es += __uint_as_float(__float_as_uint(y1) ^ shi);
            }
        }
        return es;
    };
    // the field product of the current sigma (A), both chunks (issuing lane)
    auto issue_mmas = [&]() {
#pragma unroll 1
        for (int ch = 0; ch < p.nchunk; ++ch) {
            const uint32_t d_tmem = tmem + uint32_t(ch ? p.crow[0] : 0);
            const uint32_t idesc = ch ? p.idesc[1] : p.idesc[0];
            const uint64_t bd0 = ch ? bdesc0[1] : bdesc0[0];
#pragma unroll 1
            for (int s = 0; s < ksteps; ++s)
                mma_f8f6f4(d_tmem, adesc0 + uint64_t(16 * s), bd0 + uint64_t(16 * s), idesc, s > 0 ? 1u : 0u);
            mma_commit(&bars[ch]);
        }
    };

    // ------------------------------------------------------------ cycle loop
    // J_perp level of Table 2 tracked incrementally: sub-cycle inside a tau
    // window, and the window index 0..beta inside one iteration
    const int64_t period = int64_t(a.tau) * (a.beta + 1);
    int sub = int((int64_t(a.start_cycle) % period) % a.tau);
    int lvl = int((int64_t(a.start_cycle) % period) / a.tau);
    // I0 of Eq. 6b: fixed (Table 2) or the SSA schedule of Sec. 4.4, tracked
    // the same way
    const int64_t iperiod = int64_t(p.i0_tau) * p.i0_levels;
    int isub = int((int64_t(a.start_cycle) % iperiod) % p.i0_tau);
    int ilvl = int((int64_t(a.start_cycle) % iperiod) / p.i0_tau);
    int i0cur = a.I0;
    for (int q = 0; q < ilvl; ++q) i0cur *= p.i0_mult;
    for (int it = 0; it < iters; ++it) {
        const int64_t t = int64_t(a.start_cycle) + it;
        const bool update = !kTrack || it < a.cycles;
        const bool energy = kTrack && (it > 0 || !update);
        const uint32_t parity = uint32_t(it) & 1u;
        if (*abort_flag) break;
        if (mma_warp) {
            tc_fence_after();
            if (lane == 0) issue_mmas();
            __syncwarp();
        }
        {
            const float jpf = float(a.jperp_min + lvl * a.jperp_step);
            const uint32_t JP2 = h2u(__floats2half2_rn(jpf, jpf));
            const float i0f = float(i0cur);
            const uint32_t LO2 = h2u(__floats2half2_rn(p.bias - i0f, p.bias - i0f));
            const uint32_t HI2 = h2u(__floats2half2_rn(p.bias + i0f - float(a.alpha), p.bias + i0f - float(a.alpha)));
            const uint32_t TOP2 = h2u(__floats2half2_rn(p.bias + i0f, p.bias + i0f));
            bool waited1 = false;
            auto wait_bar = [&](int ch) {
                if (!mbar_wait(&bars[ch], parity, p.wait_clocks)) {
                    *abort_flag = 1;
                    atomicExch(p.err, 1);
                }
                tc_fence_after();
            };
            // noise words of this cycle, computed while the tensor cores run.  The
            // issuing warp is busy issuing then, so warp 11 (same columns, part 2)
            // also computes its words (counter 3) and passes them on in xph.
            Philox4 ph;
            ph.x[0] = ph.x[1] = ph.x[2] = ph.x[3] = 0;
            {
                const bool helper = warp == kEpiWarps - 5;
                const int nph = mma_warp ? 0 : (helper ? 2 : 1);
#pragma unroll 1
                for (int r = 0; r < nph; ++r) {
                    Philox4 px;
                    px.x[0] = px.x[1] = px.x[2] = px.x[3] = 0;
                    if (update && valid)
                        px = philox4x32_10(uint32_t(r ? part + 1 : part), uint32_t(k), trial_g, uint32_t(t), key0, key1);
                    if (r == 0)
                        ph = px;
                    else
                        xph[lane] = make_uint4(px.x[0], px.x[1], px.x[2], px.x[3]);
                }
                if (helper) {
                    __threadfence_block();
                    bar_arrive(3, 64);
                } else if (mma_warp) {
                    bar_sync(3, 64);
                    const uint4 v = xph[lane];
                    ph.x[0] = v.x;
                    ph.x[1] = v.y;
                    ph.x[2] = v.z;
                    ph.x[3] = v.w;
                }
            }
            uint32_t newW[kMaxW];
#pragma unroll
            for (int q = 0; q < kMaxW; ++q) newW[q] = 0u;
            float esum = 0.f;
            uint32_t up_w = 0, dn_w = 0;
            // the first chunk completes first: await it once (threads with granules)
            if (gran_of(0) < p.G) wait_bar(0);
            // The second chunk's MMAs read every spin of A, so sigma(t+1) bytes of
            // granules finished before they complete wait here (only the first
            // four granule slots can lie in the first chunk, which is < 256 spins).
            uint4 pend[4];
            uint32_t pmask = 0;
            auto flush_pending = [&]() {
#pragma unroll
                for (int g2 = 0; g2 < 4; ++g2)
                    if (pmask & (1u << g2))
                        *reinterpret_cast<uint4 *>(sA + cm_off(c, gran_of(g2) * 16, Kp)) = pend[g2];
                pmask = 0;
            };
#pragma unroll
            for (int g = 0; g < kMaxG; ++g) {
                const int gg = gran_of(g);
                if (gg >= p.G) break;
                uint32_t f[kF16 ? 8 : 16];  // FP32 values, or FP16 pairs (kF16)
                // Slots >= 4 hold granules >= 16 (spins >= 256 >= the first chunk's end), so
                // the second chunk is awaited by slot 4 at the latest.
                if (g <= 4 && p.nchunk > 1 && !waited1 && gg * 16 >= p.crow[0]) {
                    wait_bar(1);
                    waited1 = true;
                    flush_pending();
                }
                if constexpr (kF16) {
                    tmem_ld16h_issue(taddr_lane + uint32_t(gg * 16), f);
                    tmem_ld_wait8(f);
                } else {
                    tmem_ld16_issue(taddr_lane + uint32_t(gg * 16), f);
                    tmem_ld_wait(f);
                }
                const int i0 = gg * 16;
                const int half = g & 1;
                const int lw = g >> 1;
                if (kShfl && update && (half == 0 || g == 0)) {
                    // sigma(t - d) of the ring neighbours, from their lanes
                    up_w = __shfl_sync(0xFFFFFFFFu, H[D][lw], src_up);
                    if (kBoth) dn_w = __shfl_sync(0xFFFFFFFFu, H[D][lw], src_dn);
                }
                // (lanes of columns beyond the last trial compute on zeros and write only
                // their own, unused rows of A; a whole trial is valid or not, so no valid
                // lane reads them)
                if constexpr (kTrack) {
                    if (energy && valid) esum = energy_add(f, H[0][lw], half, i0, esum);
                    if (!update) continue;
                }
                if (!kShfl && (half == 0 || g == 0)) {
                    up_w = slot[nb_up * p.WP + (gg >> 1)];
                    if (kBoth) dn_w = slot[nb_dn * p.WP + (gg >> 1)];
                }
                const uint32_t nw = ph.x[lw];
                uint32_t isn[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = half * 8 + q;
                    // Eq. 6a: jm*D = J sigma + h; +- n_rnd (noise); +- J_perp sigma_{k+1}(t - d)
                    uint32_t x2;
                    if constexpr (kF16)
                        x2 = f[q];
                    else
                        x2 = pack_h2(f[2 * q], f[2 * q + 1]);
                    const uint32_t n2 = ((nw << j) & kSignPair) ^ p.NR2;
                    const uint32_t c2 = ((up_w << j) & kSignPair) ^ JP2;
                    __half2 y = __hfma2(u2h(x2), u2h(p.JM2), u2h(n2));
                    y = __hadd2(y, u2h(c2));
                    if (kBoth) y = __hadd2(y, u2h(((dn_w << j) & kSignPair) ^ JP2));
                    // Eq. 6b: v = Is + I; >= I0 -> I0 - alpha; < -I0 -> -I0 (offset by bias)
                    const uint32_t ib = kFast ? __byte_perm(IsR[g][q >> 1], 0x64646464u, (q & 1) ? 0x4342 : 0x4140)
                                              : IsR[g][q];
                    const __half2 v = __hadd2(u2h(ib), y);
                    const __half2 m = __hmax2(v, u2h(LO2));
                    if (kFast) {
                        isn[q] = h2u(__hmin2(m, u2h(HI2)));
                        // Eq. 6c: sigma = +1 iff Is >= 0 iff bit 7 of the byte (bits 7 / 23)
                        const uint32_t tsh = (j <= 8) ? (isn[q] << (8 - j)) : (isn[q] >> (j - 8));
                        newW[lw] |= ~tsh & (kSignPair >> j);
                    } else {
                        const uint32_t ge = __hge2_mask(v, u2h(TOP2));
                        isn[q] = (ge & HI2) | (~ge & h2u(m));
                        IsR[g][q] = isn[q];
                        // Eq. 6c: sigma = +1 iff Is >= 0 (sign bit clear; Is is never -0)
                        newW[lw] |= (isn[q] & kSignPair) >> j;
                    }
                }
                uint4 b;
                if (kFast) {
                    uint32_t pk[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        pk[m] = __byte_perm(isn[2 * m], isn[2 * m + 1], 0x6420);
                        IsR[g][m] = pk[m];
                    }
                    b.x = (~pk[0] & 0x80808080u) | 0x38383838u;
                    b.y = (~pk[1] & 0x80808080u) | 0x38383838u;
                    b.z = (~pk[2] & 0x80808080u) | 0x38383838u;
                    b.w = (~pk[3] & 0x80808080u) | 0x38383838u;
                } else {
                    uint32_t sgn[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) sgn[q] = isn[q] & kSignPair;
                    b = fp8_bytes(sgn);
                }
                // (spins N .. N16 - 1 of a ragged granule may hold +-1 here: B is zero in
                // those K columns, so they add nothing to D)
                if (g < 4 && p.nchunk > 1 && !waited1) {
                    pend[g < 4 ? g : 0] = b;
                    pmask |= 1u << g;
                } else {
                    *reinterpret_cast<uint4 *>(sA + cm_off(c, i0, Kp)) = b;
                }
            }
            if (pmask) {
                if (!waited1) wait_bar(1);
                flush_pending();
            }
            if (energy && valid) atomicAdd(&eacc[c], static_cast<unsigned long long>(
                                                                      static_cast<long long>(esum)));
            tc_fence_before();
            // the slot path must finish every read of sigma(t - d) before any
            // owner overwrites it; energy partials must all be in eacc
            if (!kShfl || energy) bar_sync(2, kThreads);
            if (valid) {
                if (update) {
#pragma unroll
                    for (int l = D; l >= 1; --l)
#pragma unroll
                        for (int q = 0; q < kMaxW; ++q) H[l][q] = H[l - 1][q];
#pragma unroll
                    for (int q = 0; q < kMaxW; ++q) H[0][q] = newW[q];
                    if (!kShfl)
#pragma unroll
                        for (int q = 0; q < kMaxW; ++q)
                            if (gran_of(2 * q) < p.G) slot[c * p.WP + part + 4 * q] = H[D][q];
                }
                if (energy && part == 0) {
                    const long long s = static_cast<long long>(eacc[c]);
                    eacc[c] = 0ull;
                    const int64_t E = -(int64_t(p.jm) * s) / 2;
                    // E_best covers sigma(t0 + 1 .. t0 + cycles): not the start state
                    if (kTrack && it > 0 && E < e_best) {
                        e_best = E;
                        best_cycle = int32_t(t);
                    }
                    if (kTrack && it > 0 && a.e_trace)
                        a.e_trace[int64_t(it - 1) * (int64_t(a.trials) * a.R) + col0 + c] = E;
                    if (!update) e_fin = E;
                }
            }
            fence_proxy_async();
        }
        if (++sub == a.tau) {
            sub = 0;
            if (++lvl > a.beta) lvl = 0;
        }
        if (++isub == p.i0_tau) {
            isub = 0;
            if (++ilvl == p.i0_levels) {
                ilvl = 0;
                i0cur = a.I0;
            } else {
                i0cur *= p.i0_mult;
            }
        }
        bar_sync(1, kThreads);
    }

    // --------------------------------------- final energy (untracked variants)
    if constexpr (!kTrack) {
        if (need_final && !*abort_flag) {
            const uint32_t parity = uint32_t(a.cycles) & 1u;
            if (mma_warp) {
                tc_fence_after();
                if (lane == 0) issue_mmas();
                __syncwarp();
            }
            bool waited0 = false, waited1 = false;
            float esum = 0.f;
#pragma unroll
            for (int g = 0; g < kMaxG; ++g) {
                const int gg = gran_of(g);
                if (gg >= p.G) break;
                const bool ch1 = p.nchunk > 1 && gg * 16 >= p.crow[0];
                if (!(ch1 ? waited1 : waited0)) {
                    if (!mbar_wait(&bars[ch1 ? 1 : 0], parity, p.wait_clocks)) {
                        *abort_flag = 1;
                        atomicExch(p.err, 1);
                    }
                    (ch1 ? waited1 : waited0) = true;
                    tc_fence_after();
                }
                uint32_t f[kF16 ? 8 : 16];
                if constexpr (kF16) {
                    tmem_ld16h_issue(taddr_lane + uint32_t(gg * 16), f);
                    tmem_ld_wait8(f);
                } else {
                    tmem_ld16_issue(taddr_lane + uint32_t(gg * 16), f);
                    tmem_ld_wait(f);
                }
                if (valid) esum = energy_add(f, H[0][g >> 1], g & 1, gg * 16, esum);
            }
            if (valid) atomicAdd(&eacc[c], static_cast<unsigned long long>(static_cast<long long>(esum)));
            tc_fence_before();
            bar_sync(2, kThreads);
            if (valid && part == 0) e_fin = -(int64_t(p.jm) * static_cast<long long>(eacc[c])) / 2;
        }
    }

    // ---------------------------------------------------------------- outputs
    if (valid && !*abort_flag) {
        const int64_t gcol = col0 + c;
        const int64_t ht = trial0 + lt;
#pragma unroll
        for (int g = 0; g < kMaxG; ++g) {
            const int gg = gran_of(g);
            if (gg >= p.G) continue;
            const int i0 = gg * 16;
            const int lw = g >> 1;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int32_t v0, v1;
                if (kFast) {
                    const uint32_t w = IsR[g][q >> 1];
                    const int sh8 = (q & 1) * 16;
                    v0 = int32_t((w >> sh8) & 0xFFu) - 128;
                    v1 = int32_t((w >> (sh8 + 8)) & 0xFFu) - 128;
                } else {
                    const float2 v = __half22float2(u2h(IsR[g][q]));
                    v0 = int32_t(v.x);
                    v1 = int32_t(v.y);
                }
                const int i = i0 + 2 * q;
                if (i < a.N) a.Is[gcol * a.N + i] = v0;
                if (i + 1 < a.N) a.Is[gcol * a.N + i + 1] = v1;
            }
            for (int e = 0; e < 16; ++e) {
                const int i = i0 + e;
                if (i >= a.N) break;
                a.sigma[gcol * a.N + i] = word_bit(H[0][lw], uint32_t(i)) ? int8_t(-1) : int8_t(1);
                if (a.hist)
#pragma unroll
                    for (int l = 0; l < D; ++l)
                        a.hist[((ht * D + l) * a.R + k) * int64_t(a.N) + i] =
                            word_bit(H[l + 1][lw], uint32_t(i)) ? int8_t(-1) : int8_t(1);
            }
        }
        if (part == 0) {
            if (a.e_final) a.e_final[gcol] = e_fin;
            if (kTrack) {
                a.e_best[gcol] = e_best;
                a.best_cycle[gcol] = best_cycle;
            }
        }
    }
    // after an abort MMAs may still run: they complete before TMEM is freed
    if (mma_warp && lane == 0) {
        mma_commit(drain);
        mbar_wait(drain, 0u, kDrainCycles);
    }
    tc_fence_before();
    __syncthreads();
    if (mma_warp) {
        tc_fence_after();
        tmem_dealloc(tmem, p.tmem_cols);
    }
}

template <int D, bool kBoth, bool kTrack, bool kFast, bool kF16, bool kShfl>
__global__ void __launch_bounds__(kThreads, 1) ssqa_tc_kernel(const __grid_constant__ TcParams p) {
    cta_anneal<D, kBoth, kTrack, kFast, kF16, kShfl>(p, blockIdx.x);
}

// Several problems in one launch: item i owns CTAs [first[i], first[i + 1]),
// one per 128-column group of its trials, each running cta_anneal with the
// item's own parameters (instance, sizes, cycles, seed, buffers).  The items
// share the kernel variant; their shared-memory layouts fit the launch's
// dynamic size (the largest of them).
constexpr int kMaxBatch = 48;
struct TcBatch {
    int32_t count;
    int32_t first[kMaxBatch + 1];
    TcParams items[kMaxBatch];
};
static_assert(sizeof(TcBatch) <= 32764, "kernel parameters are limited to 32764 bytes");
template <int D, bool kBoth, bool kTrack, bool kFast, bool kF16, bool kShfl>
__global__ void __launch_bounds__(kThreads, 1) ssqa_tc_batch_kernel(const __grid_constant__ TcBatch b) {
    int it = 0;
    while (it + 1 < b.count && int(blockIdx.x) >= b.first[it + 1]) ++it;
    cta_anneal<D, kBoth, kTrack, kFast, kF16, kShfl>(b.items[it], int(blockIdx.x) - b.first[it]);
}

using KernelFn = void (*)(TcParams);
using BatchFn = void (*)(TcBatch);
// Batched launches exist for the shuffle-exchange variants with delay d = 1
// (Table 2's d, replica counts dividing 32); nullptr for other variants.
BatchFn pick_batch(int d, bool both, bool track, bool bytes, bool f16, bool shfl);

// Kernel variants are split over several translation units (per delay d, and
// shuffle vs shared-memory-slot exchange) so that they compile in parallel.
// f16: FP16 accumulator (byte counters only).
KernelFn pick_shfl_d0(bool both, bool track, bool f16);
KernelFn pick_shfl_d1(bool both, bool track, bool f16);
KernelFn pick_shfl_d2(bool both, bool track, bool f16);
KernelFn pick_shfl_d3(bool both, bool track, bool f16);
KernelFn pick_slot_d0(bool both, bool track, bool bytes, bool f16);
KernelFn pick_slot_d1(bool both, bool track, bool bytes, bool f16);
KernelFn pick_slot_d2(bool both, bool track, bool bytes, bool f16);
KernelFn pick_slot_d3(bool both, bool track, bool bytes, bool f16);

#define SSQA_TC_PICK_TRACK(DD, B, F, H, S) \
    (track ? ssqa_tc_kernel<DD, B, true, F, H, S> : ssqa_tc_kernel<DD, B, false, F, H, S>)
#define SSQA_TC_DEFINE_PICK_SHFL(DD)                                                                   \
    KernelFn pick_shfl_d##DD(bool both, bool track, bool f16) {                                         \
        if (f16) return both ? SSQA_TC_PICK_TRACK(DD, true, true, true, true)                          \
                             : SSQA_TC_PICK_TRACK(DD, false, true, true, true);                        \
        return both ? SSQA_TC_PICK_TRACK(DD, true, true, false, true) : SSQA_TC_PICK_TRACK(DD, false, true, false, true); \
    }
#define SSQA_TC_DEFINE_PICK_SLOT(DD)                                                                   \
    KernelFn pick_slot_d##DD(bool both, bool track, bool bytes, bool f16) {                             \
        if (bytes && f16) return both ? SSQA_TC_PICK_TRACK(DD, true, true, true, false)                \
                                      : SSQA_TC_PICK_TRACK(DD, false, true, true, false);              \
        if (bytes) return both ? SSQA_TC_PICK_TRACK(DD, true, true, false, false)                      \
                               : SSQA_TC_PICK_TRACK(DD, false, true, false, false);                    \
        return both ? SSQA_TC_PICK_TRACK(DD, true, false, false, false)                                \
                    : SSQA_TC_PICK_TRACK(DD, false, false, false, false);                              \
    }

}  // namespace tc
}  // namespace ssqa
