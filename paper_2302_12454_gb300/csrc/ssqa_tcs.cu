// Streamed tensor-core path of SSQA for sm_103a, for instances whose
// operands do not fit in one SM (N > 400).
//
// A CTA owns one group of 128 spin columns (whole trials, as in the resident
// kernel), or two groups in dual mode, and a share of the spin chunks (256
// spins each) of the field product
//   D[c][i] = sum_j sigma_{j,c}(t) J_ij / jm + h_i / jm     (Eq. 6a, exact FP8)
// A thread-block cluster of CS CTAs covers all chunks of its column group(s);
// chunk ch belongs to cluster rank ch mod CS.  Per cycle:
//   producer warp  streams, for each owned chunk, the K-blocks of A (sigma(t)
//                  of 128 columns, 4 KB per group and K-block) and B (J rows
//                  of the chunk, 8 KB per K-block) from L2 into a shared-memory
//                  ring whose stages hold kps consecutive K-blocks, one bulk
//                  async copy per operand and stage (consecutive K-blocks are
//                  contiguous in both images), completing on mbarriers;
//   MMA warp       issues per K-block one tcgen05.mma kind::f8f6f4 (M 128,
//                  N <= 256, K 32) per group, all groups on the same B block;
//   epilogue warps (8; 16 in dual mode) turn finished accumulators into
//                  sigma(t+1) of the chunk (Eq. 6a-6c, the same packed-half2
//                  arithmetic as the resident kernel): in single mode while
//                  the next chunk's MMAs run into the other of two TMEM
//                  buffers, in dual mode (one buffer per group) before them;
// and a cluster barrier closes the cycle.  sigma lives in L2 as FP8 operand
// blocks, one slot per history level (the replica term reads the ring
// neighbour's sigma(t - d) from its slot), and the counters as bytes Is + 128.
// Dual mode carries a third fewer operand bytes per MAC; the host takes it
// for chunks of at least 160 K-blocks, where the MMAs of a chunk outlast its
// epilogue by far.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <utility>

#include "ssqa_tc_kernel.cuh"

namespace ssqa {
namespace tcs {
using namespace tc;

// A bulk copy's delivery rate into an SM grows with the bytes it keeps in
// flight (~75 B/clk with about 192 KB outstanding, ~23 with one 12 KB stage of
// one K-block) and with the size of each copy: at N = 2500 (single mode) three
// stages of 6 K-blocks (72 KB, one 24 KB and one 48 KB copy each) anneal in
// 0.227 s, four of 4 K-blocks in 0.254 s, six of 3 in 0.286 s (two of 9: 0.224 s,
// within the run-to-run spread, with no stage left to overlap a refill).  Dual mode keeps
// three stages of 4 K-blocks (64 KB each; two stages of 6 took 0.311 s instead
// of 0.268 s on SK N = 8192).
constexpr int kABytes = 128 * 32;   // one K-block of A
constexpr int kBBytes = 256 * 32;   // one K-block of a B chunk
template <bool kDual> __host__ __device__ constexpr int stage_kblocks() { return kDual ? 4 : 6; }
constexpr int kRingStages = 3;      // ring stages in both modes
// dual mode: A of both column groups and one B run; single mode: A and B runs
template <bool kDual> __host__ __device__ constexpr int stage_bytes() {
    return stage_kblocks<kDual>() * ((kDual ? 2 : 1) * kABytes + kBBytes);
}
// Epilogue warps: 8 (2 per TMEM lane quadrant) in single mode, where a
// chunk's epilogue hides under the next chunk's MMAs and 168 registers a
// thread leave the prefetched loads unspilled; 16 (4 per quadrant) in dual
// mode, where the MMAs wait for the epilogue (SK N = 8192: 0.357 s instead of
// 0.39 s per anneal; 18 warps on four schedulers allow 96 registers).
template <bool kDual> __host__ __device__ constexpr int epi_warps() { return kDual ? 16 : 8; }
template <bool kDual> __host__ __device__ constexpr int cta_threads() { return (2 + epi_warps<kDual>()) * 32; }

struct SParams {
    AnnealArgs a;
    const uint8_t *B;       // [NCH][KB][256 x 32] blocks
    uint8_t *A;             // [groups][L][KB][128 x 32] blocks
    uint8_t *IsB;           // [Np / 16][cols][16] counters + 128 (a warp's 16-byte loads are contiguous)
    const float *hf;        // h / jm as float (N)
    unsigned long long *eacc;  // [2][cols]
    int64_t *ebest, *efin;     // [cols]
    int32_t *bcyc;             // [cols]
    int *err;
    int32_t N16, KB, NCH, L, CS, Tb, jm, last_rows;
    int32_t dual;           // a CTA serves two column groups (one accumulator buffer each)
    long long wait_clocks;  // bound of every wait for copies, MMAs or other warps (SM clocks)
    uint32_t NR2, JM2;
    float bias;
    int32_t i0_levels, i0_mult, i0_tau;
};

// --------------------------------------------------------------- PTX helpers
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Byte offset of (row r, k) inside one 32-byte-wide K-block (core matrices).
__device__ __forceinline__ uint32_t blk_off(int r, int k) {
    return uint32_t((r >> 3) * 256 + ((k >> 4) & 1) * 128 + (r & 7) * 16 + (k & 15));
}
__device__ __forceinline__ int64_t slot_of(int64_t t, int32_t L) { return ((t % L) + L) % L; }

// ------------------------------------------------------------------- kernel
template <bool kTrack, bool kDual>
__global__ void __launch_bounds__(cta_threads<kDual>(), 1) ssqa_tcs_kernel(const __grid_constant__ SParams p) {
    constexpr int kEpi = epi_warps<kDual>();
    constexpr int kParts = kEpi / 4;    // epilogue warps per TMEM lane quadrant
    constexpr int kPairs = 4 / kParts;  // word pairs (w, w + 4) of a chunk per thread
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *ring = sm;
    // stage = A run of group 0 [kps][128 x 32], (dual) A run of group 1, then
    // the B run [kps][256 x 32]
    constexpr int kKps = stage_kblocks<kDual>();
    constexpr int kStages = kRingStages;
    constexpr int sbytes = stage_bytes<kDual>();
    constexpr int a2off = kKps * kABytes;
    constexpr int boff = (kDual ? 2 : 1) * kKps * kABytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + kStages * sbytes);
    uint64_t *empty = full + kStages;
    uint64_t *tfull = empty + kStages;   // [2]
    uint64_t *tempty = tfull + 2;        // [2]
    uint64_t *drain = tempty + 2;        // [1]
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 1);

    const AnnealArgs &a = p.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rank = int(cluster_rank());
    // Dual mode: column groups 2 pg and 2 pg + 1 (the second may not exist),
    // whose MMAs share each B block, one TMEM accumulator per group.  Single
    // mode: one group, its accumulator double-buffered across chunks so that
    // a chunk's epilogue overlaps the next chunk's MMAs.
    const int64_t ngroups = (int64_t(a.trials) + p.Tb - 1) / p.Tb;
    const int64_t grp0 = (kDual ? 2 : 1) * int64_t(blockIdx.x / p.CS);
    const int ng = kDual && grp0 + 1 < ngroups ? 2 : 1;
    const bool need_final = a.e_final != nullptr || kTrack;
    const int iters = a.cycles + (need_final ? 1 : 0);
    const int nmine = (p.NCH - rank + p.CS - 1) / p.CS;  // chunks rank, rank + CS, ...
    const int64_t cols = int64_t(a.trials) * a.R;
    const int64_t slot_stride = int64_t(p.L) * p.KB * kABytes;  // one group's operand slots
    uint8_t *Ag0 = p.A + grp0 * slot_stride;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpi);
        }
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_holder, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    // A failed bounded wait (or the flag set by another CTA) stops all work;
    // every thread still passes every cluster barrier, so the exit is uniform.
    bool abort_run = false;
    uint32_t nis = 0;  // producer: stage fills issued

    // pipeline positions carried across cycles
    int ps = 0, pph = 1;   // producer: stage, empty-barrier parity (first pass free)
    int ms = 0, mph = 0;   // MMA: stage, full-barrier parity
    uint32_t mt_ph = 3u;   // MMA: tmem-empty parity per buffer (bit b)
    uint32_t et_ph = 0u;   // epilogue: tmem-full parity per buffer (bit b)

    // epilogue identity: TMEM lane quadrant qd (column c of each group), part
    // 0 .. kParts - 1 of the words; accumulators at TMEM column 256 gi (dual mode,
    // group gi) or 256 (m & 1) (single mode, the CTA's m-th chunk)
    const int ew = warp - 2;
    const int qd = warp & 3, part = ew >> 2;
    const int c = qd * 32 + lane;
    auto vcols_of = [&](int gi) -> int {
        const int64_t tr0 = (grp0 + gi) * p.Tb;
        return int((a.trials - tr0 < p.Tb ? a.trials - tr0 : p.Tb) * a.R);
    };
    const bool valid0 = warp >= 2 && c < vcols_of(0);
    const bool valid1 = kDual && warp >= 2 && ng > 1 && c < vcols_of(1);
    const int lt = valid0 ? c / a.R : 0, k = valid0 ? c % a.R : 0;
    const int nb_up = lt * a.R + (k + 1) % a.R;
    const int nb_dn = lt * a.R + (k + a.R - 1) % a.R;
    const int64_t gcol0 = grp0 * p.Tb * a.R + c;
    const int64_t gcol1 = gcol0 + int64_t(p.Tb) * a.R;
    int64_t e_best0 = LLONG_MAX, e_best1 = LLONG_MAX;
    int32_t best_cycle0 = -1, best_cycle1 = -1;

    const int64_t period = int64_t(a.tau) * (a.beta + 1);
    int sub = int((int64_t(a.start_cycle) % period) % a.tau);
    int lvl = int((int64_t(a.start_cycle) % period) / a.tau);
    const int64_t iperiod = int64_t(p.i0_tau) * p.i0_levels;
    int isub = int((int64_t(a.start_cycle) % iperiod) % p.i0_tau);
    int ilvl = int((int64_t(a.start_cycle) % iperiod) / p.i0_tau);
    int i0cur = a.I0;
    for (int q = 0; q < ilvl; ++q) i0cur *= p.i0_mult;

    for (int it = 0; it < iters; ++it) {
        const int64_t t = int64_t(a.start_cycle) + it;
        const bool update = it < a.cycles;
        const bool energy = (kTrack && it > 0) || !update;
        const int64_t cur_off = slot_of(t, p.L) * p.KB * kABytes;  // sigma(t) slot of a group
        if (*reinterpret_cast<volatile int *>(p.err)) abort_run = true;
        if (warp == 0) {
            // ---------------------------------------------------- producer
            if (lane == 0 && !abort_run) {
                fence_async_global();
                for (int m = 0; m < nmine && !abort_run; ++m) {
                    const int ch = rank + m * p.CS;
                    const uint8_t *Bc = p.B + int64_t(ch) * p.KB * kBBytes;
                    if (m > 0 && *reinterpret_cast<volatile int *>(p.err)) abort_run = true;
                    for (int kb = 0; kb < p.KB && !abort_run; kb += kKps) {
                        const int nkb = p.KB - kb < kKps ? p.KB - kb : kKps;
                        if (!mbar_wait(&empty[ps], uint32_t(pph), p.wait_clocks)) {
                            atomicExch(p.err, 1);
                            abort_run = true;
                            break;
                        }
                        // nkb K-blocks: A of each group, then the B run both groups' MMAs share
                        uint8_t *st = ring + ps * sbytes;
                        mbar_expect_tx(&full[ps], uint32_t(nkb * (ng * kABytes + kBBytes)));
                        bulk_g2s(st, Ag0 + cur_off + int64_t(kb) * kABytes, uint32_t(nkb * kABytes), &full[ps]);
                        if (kDual && ng > 1)
                            bulk_g2s(st + a2off, Ag0 + slot_stride + cur_off + int64_t(kb) * kABytes,
                                     uint32_t(nkb * kABytes), &full[ps]);
                        bulk_g2s(st + boff, Bc + int64_t(kb) * kBBytes, uint32_t(nkb * kBBytes), &full[ps]);
                        ++nis;
                        if (++ps == kStages) {
                            ps = 0;
                            pph ^= 1;
                        }
                    }
                }
            }
            __syncwarp();
        } else if (warp == 1) {
            // ------------------------------------------------------- MMA
            if (lane == 0 && !abort_run) {
                for (int m = 0; m < nmine && !abort_run; ++m) {
                    const int ch = rank + m * p.CS;
                    const int b = kDual ? 0 : (m & 1);  // accumulator buffer
                    const int rows = ch == p.NCH - 1 ? p.last_rows : 256;
                    const uint32_t idesc = (1u << 4) | (uint32_t(rows >> 3) << 17) | (uint32_t(128 >> 4) << 24);
                    if (m > 0 && *reinterpret_cast<volatile int *>(p.err)) abort_run = true;
                    // the epilogue has read this buffer's previous accumulators
                    if (abort_run || !mbar_wait(&tempty[b], (mt_ph >> b) & 1u, p.wait_clocks)) {
                        if (!abort_run) atomicExch(p.err, 1);
                        abort_run = true;
                        break;
                    }
                    mt_ph ^= 1u << b;
                    tc_fence_after();
                    for (int kb = 0; kb < p.KB; kb += kKps) {
                        const int nkb = p.KB - kb < kKps ? p.KB - kb : kKps;
                        if (!mbar_wait(&full[ms], uint32_t(mph), p.wait_clocks)) {
                            atomicExch(p.err, 1);
                            abort_run = true;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t st = smem_u32(ring + ms * sbytes);
                        for (int j = 0; j < nkb; ++j) {
                            const uint32_t acc = kb + j > 0 ? 1u : 0u;
                            const uint64_t bd = smem_desc(st + uint32_t(boff + j * kBBytes), 128u, 256u);
                            mma_f8f6f4(tmem + uint32_t(b * 256), smem_desc(st + uint32_t(j * kABytes), 128u, 256u), bd,
                                       idesc, acc);
                            if (kDual && ng > 1)
                                mma_f8f6f4(tmem + 256u, smem_desc(st + uint32_t(a2off + j * kABytes), 128u, 256u), bd,
                                           idesc, acc);
                        }
                        mma_commit(&empty[ms]);  // frees the stage when these MMAs complete
                        if (++ms == kStages) {
                            ms = 0;
                            mph ^= 1;
                        }
                    }
                    if (abort_run) break;
                    mma_commit(&tfull[b]);
                }
            }
            __syncwarp();
        } else {
            // -------------------------------------------------- epilogue
            abort_run = __any_sync(0xffffffffu, abort_run);
            const float jpf = float(a.jperp_min + lvl * a.jperp_step);
            const uint32_t JP2 = h2u(__floats2half2_rn(jpf, jpf));
            const float i0f = float(i0cur);
            const uint32_t LO2 = h2u(__floats2half2_rn(p.bias - i0f, p.bias - i0f));
            const uint32_t HI2 = h2u(__floats2half2_rn(p.bias + i0f - float(a.alpha), p.bias + i0f - float(a.alpha)));
            const uint32_t TOP2 = h2u(__floats2half2_rn(p.bias + i0f, p.bias + i0f));
            const int64_t old_off = slot_of(t - a.delay, p.L) * p.KB * kABytes;
            const int64_t next_off = slot_of(t + 1, p.L) * p.KB * kABytes;
            long long esum0 = 0, esum1 = 0;
            for (int m = 0; m < nmine && !abort_run; ++m) {
                const int ch = rank + m * p.CS;
                const int b = kDual ? 0 : (m & 1);
#pragma unroll 1
                for (int gi = 0; gi < (kDual ? ng : 1); ++gi) {
                // group gi: its columns, operand slots, counters and noise
                const bool valid = gi ? valid1 : valid0;
                const int64_t trial0 = (grp0 + gi) * p.Tb;
                const uint32_t trial_g = a.trial_offset + uint32_t(trial0 + lt);
                const int64_t gcol = trial0 * a.R + c;
                uint8_t *Ag = Ag0 + gi * slot_stride;
                const uint8_t *Acur = Ag + cur_off;
                const uint8_t *Aold = Ag + old_off;
                uint8_t *Anext = Ag + next_off;
                long long esum = 0;
                // This thread's words of the chunk: the kPairs pairs (w, w + 4), w =
                // 8 ch + kPairs part + j.  The words of a pair share one Philox call (same
                // counter), made before the MMAs are awaited; the output of word w is
                // (w / 4) % 4 = 2 (ch % 2) for w and 2 (ch % 2) + 1 for w + 4.
                const int wbase = 8 * ch + kPairs * part;
                uint32_t nq[2 * kPairs];
#pragma unroll
                for (int j = 0; j < 2 * kPairs; ++j) nq[j] = 0;
                if (update) {
                    const bool odd = ch & 1;
#pragma unroll
                    for (int j = 0; j < kPairs; ++j) {
                        const Philox4 ph = philox4x32_10(noise_ctr(uint32_t(wbase + j)), uint32_t(k), trial_g,
                                                         uint32_t(t), uint32_t(a.seed), uint32_t(a.seed >> 32));
                        nq[2 * j] = odd ? ph.x[2] : ph.x[0];
                        nq[2 * j + 1] = odd ? ph.x[3] : ph.x[1];
                    }
                }
                // Granule g of the chunk (q = g / 2, hh = g % 2): spins i0 .. i0 + 15 of
                // word wbase + q / 2 + 4 (q % 2), noise word nq[q].  Its counters and its
                // upper ring neighbour's sigma(t - d) do not depend on this cycle's MMAs;
                // in single mode all the thread's granules' values are loaded before the
                // accumulator is awaited, so that their L2 latencies overlap the wait and
                // each other.
                constexpr int kGran = 4 * kPairs;
                auto gran_i0 = [&](int g) { return 32 * (wbase + 4 * ((g >> 1) & 1) + (g >> 2)) + 16 * (g & 1); };
                auto is_ptr = [&](int i0) { return p.IsB + (int64_t(i0 >> 4) * cols + gcol) * 16; };
                auto nu_ptr = [&](int i0) { return Aold + int64_t(i0 >> 5) * kABytes + blk_off(nb_up, i0 & 31); };
                auto gran_loads = [&](int g, uint4 &isv, uint4 &nu) {
                    const int i0 = gran_i0(g);
                    if (update && valid && i0 < p.N16) {
                        isv = *reinterpret_cast<const uint4 *>(is_ptr(i0));
                        nu = *reinterpret_cast<const uint4 *>(nu_ptr(i0));
                    } else {
                        isv = make_uint4(0, 0, 0, 0);
                        nu = isv;
                    }
                };
                uint4 pis[kDual ? 1 : kGran], pnu[kDual ? 1 : kGran];
                if constexpr (!kDual) {
#pragma unroll
                    for (int g = 0; g < kGran; ++g) gran_loads(g, pis[g], pnu[g]);
                }
                if (gi == 0) {  // the chunk's accumulators (of both groups)
                    const bool ok = mbar_wait(&tfull[b], (et_ph >> b) & 1u, p.wait_clocks);
                    if (__any_sync(0xffffffffu, !ok)) {
                        if (lane == 0) atomicExch(p.err, 1);
                        abort_run = true;
                        break;
                    }
                    et_ph ^= 1u << b;
                    tc_fence_after();
                }
                auto granule = [&](int g, const uint4 isv, const uint4 nu) {
                    const int q = g >> 1, hh = g & 1;
                    const int i0 = gran_i0(g);
                    if (i0 >= p.N16) return;  // warp-uniform
                    uint32_t nw = nq[0];  // nq[q] by selects (g is a loop variable in dual mode)
#pragma unroll
                    for (int j = 1; j < 2 * kPairs; ++j)
                        if (q == j) nw = nq[j];
                    uint32_t f[16];
                    __syncwarp();
                    tmem_ld16_issue(tmem + (uint32_t(qd * 32) << 16) + uint32_t((b + gi) * 256 + (i0 - 256 * ch)), f);
                    tmem_ld_wait(f);
                    if (!valid) return;
                    const int kb = i0 >> 5;
                    const uint32_t ob = blk_off(c, i0 & 31);
                    if (energy) {
                        // sigma_i (D_i + h_i / jm) = sigma_i (sum_j J_ij sigma_j + 2 h_i) / jm; a
                        // 16-spin partial sum is an exact float (|terms| <= 2^15)
                        const uint4 so = *reinterpret_cast<const uint4 *>(Acur + int64_t(kb) * kABytes + ob);
                        const uint32_t sw[4] = {so.x, so.y, so.z, so.w};
                        float tsum = 0.f;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int i = i0 + e;
                            if (i >= a.N) break;
                            const float y = __uint_as_float(f[e]) + __ldg(&p.hf[i]);
                            const uint32_t sgn = (sw[e >> 2] << (24 - 8 * (e & 3))) & 0x80000000u;
                            tsum += __uint_as_float(__float_as_uint(y) ^ sgn);
                        }
                        esum += static_cast<long long>(tsum);
                        if (!update) return;
                    }
                    // ring neighbours' sigma(t - d) (FP8 bytes, sign bit 7)
                    const uint32_t nuw[4] = {nu.x, nu.y, nu.z, nu.w};
                    uint32_t ndw[4] = {0, 0, 0, 0};
                    if (a.both) {
                        const uint4 nd = *reinterpret_cast<const uint4 *>(Aold + int64_t(kb) * kABytes +
                                                                          blk_off(nb_dn, i0 & 31));
                        ndw[0] = nd.x;
                        ndw[1] = nd.y;
                        ndw[2] = nd.z;
                        ndw[3] = nd.w;
                    }
                    const uint32_t isw[4] = {isv.x, isv.y, isv.z, isv.w};
                    uint32_t isn[8];
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        const int j = hh * 8 + qq;
                        const uint32_t x2 = pack_h2(f[2 * qq], f[2 * qq + 1]);
                        const uint32_t n2 = ((nw << j) & kSignPair) ^ p.NR2;
                        // bytes 2qq, 2qq+1 of the neighbour row: signs to bits 15 / 31
                        const uint32_t sel = (qq & 1) ? 0x3727 : 0x1707;
                        const uint32_t c2 = (__byte_perm(nuw[qq >> 1], 0, sel) & kSignPair) ^ JP2;
                        __half2 y = __hfma2(u2h(x2), u2h(p.JM2), u2h(n2));
                        y = __hadd2(y, u2h(c2));
                        if (a.both)
                            y = __hadd2(y, u2h((__byte_perm(ndw[qq >> 1], 0, sel) & kSignPair) ^ JP2));
                        const uint32_t ib = __byte_perm(isw[qq >> 1], 0x64646464u, (qq & 1) ? 0x4342 : 0x4140);
                        const __half2 v = __hadd2(u2h(ib), y);
                        const __half2 mm = __hmax2(v, u2h(LO2));
                        const uint32_t ge = __hge2_mask(v, u2h(TOP2));
                        isn[qq] = (ge & HI2) | (~ge & h2u(mm));
                    }
                    uint32_t pk[4];
#pragma unroll
                    for (int mq = 0; mq < 4; ++mq) pk[mq] = __byte_perm(isn[2 * mq], isn[2 * mq + 1], 0x6420);
                    *reinterpret_cast<uint4 *>(is_ptr(i0)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    uint4 bo;
                    bo.x = (~pk[0] & 0x80808080u) | 0x38383838u;
                    bo.y = (~pk[1] & 0x80808080u) | 0x38383838u;
                    bo.z = (~pk[2] & 0x80808080u) | 0x38383838u;
                    bo.w = (~pk[3] & 0x80808080u) | 0x38383838u;
                    if (i0 + 16 > a.N) bo = mask_tail(bo, i0, a.N);
                    *reinterpret_cast<uint4 *>(Anext + int64_t(kb) * kABytes + ob) = bo;
                };
                if constexpr (!kDual) {
#pragma unroll
                    for (int g = 0; g < kGran; ++g) granule(g, pis[g], pnu[g]);
                } else {
#pragma unroll 1
                    for (int g = 0; g < kGran; ++g) {
                        uint4 isv, nu;
                        gran_loads(g, isv, nu);
                        granule(g, isv, nu);
                    }
                }
                if (gi)
                    esum1 += esum;
                else
                    esum0 += esum;
                }
                if (abort_run) break;
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
            }
            if (energy && valid0 && !abort_run)
                atomicAdd(&p.eacc[(it & 1) * cols + gcol0], static_cast<unsigned long long>(esum0));
            if (energy && valid1 && !abort_run)
                atomicAdd(&p.eacc[(it & 1) * cols + gcol1], static_cast<unsigned long long>(esum1));
            fence_async_global();
        }
        // ------------------------------------------------------ cycle end
        cluster_sync();
        if (energy && rank == 0 && part == 0) {
#pragma unroll
            for (int gi = 0; gi < 2; ++gi) {
                if (!(gi ? valid1 : valid0)) continue;
                const int64_t gcol = gi ? gcol1 : gcol0;
                const long long s = static_cast<long long>(atomicExch(&p.eacc[(it & 1) * cols + gcol], 0ull));
                const int64_t E = -(int64_t(p.jm) * s) / 2;
                int64_t &eb = gi ? e_best1 : e_best0;
                if (kTrack && it > 0 && E < eb) {
                    eb = E;
                    (gi ? best_cycle1 : best_cycle0) = int32_t(t);
                }
                if (kTrack && it > 0 && a.e_trace) a.e_trace[int64_t(it - 1) * cols + gcol] = E;
                if (!update && p.efin) p.efin[gcol] = E;
            }
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
    }
    if (kTrack && rank == 0 && part == 0) {
        if (valid0) {
            p.ebest[gcol0] = e_best0;
            p.bcyc[gcol0] = best_cycle0;
        }
        if (valid1) {
            p.ebest[gcol1] = e_best1;
            p.bcyc[gcol1] = best_cycle1;
        }
    }
    // Drain before exit: the producer waits (bounded) for its last copy into
    // every stage, the MMA thread for all MMAs it issued.
    if (warp == 0 && lane == 0) {
        for (int s = 0; s < kStages && uint32_t(s) < nis; ++s) {
            const uint32_t last = (nis - 1u - uint32_t(s)) / uint32_t(kStages);
            mbar_wait(&full[s], last & 1u, kDrainCycles);
        }
    }
    if (warp == 1 && lane == 0) {
        mma_commit(drain);
        mbar_wait(drain, 0u, kDrainCycles);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    cluster_sync();
}

// Initial operand slots and counters: sigma(t0 - l) for l = 0..d, the h
// weight columns in every slot, zero elsewhere; counters Is + 128.
__global__ void tcs_init_kernel(SParams p, const uint8_t *a_w, int nh) {
    const AnnealArgs &a = p.a;
    const int64_t groups = (int64_t(a.trials) + p.Tb - 1) / p.Tb;
    const int64_t per_slot = int64_t(p.KB) * kABytes;
    const int64_t total = groups * p.L * per_slot;
    const int64_t t0 = a.start_cycle;
    for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < total; x += int64_t(gridDim.x) * blockDim.x) {
        const int64_t g = x / (p.L * per_slot);
        const int64_t rem = x % (p.L * per_slot);
        const int s = int(rem / per_slot);
        const int64_t inb = rem % per_slot;
        const int kb = int(inb / kABytes);
        const int off = int(inb % kABytes);
        // invert blk_off: off = (r/8)*256 + kc*128 + (r%8)*16 + e
        const int r = (off >> 8) * 8 + ((off >> 4) & 7);
        const int kk = kb * 32 + ((off >> 7) & 1) * 16 + (off & 15);
        const int64_t trial = g * p.Tb + r / a.R;
        const bool vr = r < p.Tb * a.R && trial < a.trials;
        uint8_t v = 0;
        if (vr) {
            const int kr = r % a.R;
            const int64_t col = trial * a.R + kr;
            if (kk >= p.N16 && kk < p.N16 + nh) {
                v = a_w[kk - p.N16];
            } else if (kk < a.N) {
                // which history level is slot s?  level l with slot(t0 - l) == s
                int lev = -1;
                for (int l = 0; l <= a.delay; ++l)
                    if (slot_of(t0 - l, p.L) == s) lev = l;
                if (lev >= 0) {
                    int8_t sg;
                    if (a.init_mode == SSQA_INIT_FROM_STATE) {
                        sg = lev == 0 ? a.sigma[col * a.N + kk]
                                      : a.hist[((trial * a.delay + (lev - 1)) * a.R + kr) * int64_t(a.N) + kk];
                    } else if (a.init_mode == SSQA_INIT_RANDOM) {
                        const uint32_t w = noise_word(a.seed, uint32_t(kk), uint32_t(kr), a.trial_offset + uint32_t(trial),
                                                      0xFFFFFFFFu);
                        sg = ((w >> spin_bit_pos(uint32_t(kk))) & 1u) ? int8_t(-1) : int8_t(1);
                    } else {
                        sg = -1;
                    }
                    v = sg < 0 ? 0xB8 : 0x38;
                }
            }
        }
        p.A[x] = v;
    }
    const int64_t cols = int64_t(a.trials) * a.R;
    for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < cols * a.Np;
         x += int64_t(gridDim.x) * blockDim.x) {
        // x = ((i / 16) * cols + col) * 16 + i % 16
        const int64_t col = (x / 16) % cols;
        const int i = int((x / (16 * cols)) * 16 + x % 16);
        int v = 0;
        if (i < a.N && a.init_mode == SSQA_INIT_FROM_STATE) v = a.Is[col * a.N + i];
        if (v < -128 || v > 127) {
            atomicExch(p.err, 2);  // the byte counters cannot hold this state
            v = 0;
        }
        p.IsB[x] = uint8_t(v + 128);
    }
    for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < 2 * cols; x += int64_t(gridDim.x) * blockDim.x)
        p.eacc[x] = 0ull;
}

// Results: sigma(tf), history, counters (the energies are written by the kernel).
__global__ void tcs_finish_kernel(SParams p, int64_t tf) {
    const AnnealArgs &a = p.a;
    const int64_t cols = int64_t(a.trials) * a.R;
    for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < cols * a.N; x += int64_t(gridDim.x) * blockDim.x) {
        const int64_t col = x / a.N;
        const int i = int(x % a.N);
        const int64_t trial = col / a.R;
        const int kr = int(col % a.R);
        const int64_t g = trial / p.Tb;
        const int r = int((trial % p.Tb) * a.R + kr);
        const uint8_t *Ag = p.A + g * int64_t(p.L) * p.KB * kABytes;
        const int64_t o = int64_t(i >> 5) * kABytes + blk_off(r, i & 31);
        a.sigma[x] = (Ag[slot_of(tf, p.L) * p.KB * kABytes + o] & 0x80) ? int8_t(-1) : int8_t(1);
        if (a.hist)
            for (int l = 0; l < a.delay; ++l)
                a.hist[((trial * a.delay + l) * a.R + kr) * int64_t(a.N) + i] =
                    (Ag[slot_of(tf - 1 - l, p.L) * p.KB * kABytes + o] & 0x80) ? int8_t(-1) : int8_t(1);
        a.Is[x] = int32_t(p.IsB[(int64_t(i >> 4) * cols + col) * 16 + (i & 15)]) - 128;
    }
}

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

void configure_once(void (*fn)(SParams), int smem) {
    static std::mutex mu;
    static std::set<std::pair<int, void (*)(SParams)>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, fn})) return;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, int(cudaSharedmemCarveoutMaxShared));
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin > smem ? optin : smem);
    cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    done.insert({dev, fn});
}

}  // namespace tcs

bool tcs_supported(const TcImage &img, const AnnealArgs &a, std::string *why) {
    if (!img.s_ok) {
        *why = img.why.empty() ? "no streamed operand image (N <= 256 or too many h digits)" : img.why;
        return false;
    }
    if (img.nh > 16) {
        *why = "too many h digit columns";
        return false;
    }
    if (a.R > 128) {
        *why = "R > 128";
        return false;
    }
    const int64_t jpmax = std::max<int64_t>(std::llabs(int64_t(a.jperp_min)),
                                            std::llabs(int64_t(a.jperp_min) + int64_t(a.jperp_step) * a.beta));
    const int64_t i0_top = a.i0_max > a.I0 ? a.i0_max : a.I0;
    if (i0_top > 127) {
        *why = "counters above 127 do not fit the byte state of the streamed path";
        return false;
    }
    if (i0_top + a.n_rnd + (a.both ? 2 : 1) * jpmax > 1024) {
        *why = "I0 + n_rnd + |J_perp| terms exceed the exact FP16 epilogue range (1024)";
        return false;
    }
    return true;
}

namespace {
struct LaunchCfg {
    void (*fn)(tcs::SParams);
    int threads, smem;
};
LaunchCfg launch_cfg(bool dual, bool track) {
    using namespace tcs;
    LaunchCfg c;
    c.fn = track ? (dual ? ssqa_tcs_kernel<true, true> : ssqa_tcs_kernel<true, false>)
                 : (dual ? ssqa_tcs_kernel<false, true> : ssqa_tcs_kernel<false, false>);
    c.threads = dual ? cta_threads<true>() : cta_threads<false>();
    c.smem = kRingStages * (dual ? stage_bytes<true>() : stage_bytes<false>()) + 1024 + 512;  // ring, alignment, barriers
    return c;
}
}  // namespace

int tcs_cluster_size(const TcImage &img, const AnnealArgs &a, int nsm) {
    const int64_t Tb = 128 / a.R;
    const int64_t groups = (int64_t(a.trials) + Tb - 1) / Tb;
    const bool dual = img.KB >= 160;
    const int64_t clusters = dual ? (groups + 1) / 2 : groups;  // one per column group (pair), CTAs per chunk rank
    // A cycle takes as long as the rank with the most chunks.  Take the
    // smallest cluster that reaches the fewest chunks per rank among those
    // whose clusters all fit on the device at once, up to 16 CTAs (a
    // non-portable size): SK N = 8192 runs 8 clusters of 11 ranks with at most
    // 3 chunks each in 0.27 s, against 8 ranks of 4 chunks in 0.35 s; 16 ranks
    // of 2 do not all fit.  N = 2500: 2 ranks of 5 chunks (3 would need 192 SMs).
    // Without a device, portable sizes (<= 8) are assumed to fit.
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    const LaunchCfg lc = launch_cfg(dual, a.track_best);
    static std::mutex mu;
    static std::map<std::tuple<int, void (*)(tcs::SParams), int64_t, int, int>, int> memo;
    const auto key = std::make_tuple(dev, lc.fn, clusters, img.NCH, nsm);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
    }
    if (dev >= 0) tcs::configure_once(lc.fn, lc.smem);
    int best = 1, best_chunks = img.NCH;
    for (int cs = 2; cs <= 16 && cs <= img.NCH; ++cs) {
        const int chunks = (img.NCH + cs - 1) / cs;
        if (chunks >= best_chunks) continue;
        if (clusters * cs > nsm) break;
        if (dev >= 0) {
            cudaLaunchConfig_t cfg{};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = unsigned(cs);
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(unsigned(clusters * cs), 1, 1);
            cfg.blockDim = dim3(unsigned(lc.threads), 1, 1);
            cfg.dynamicSmemBytes = size_t(lc.smem);
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclus = 0;
            if (cudaOccupancyMaxActiveClusters(&nclus, lc.fn, &cfg) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (nclus < clusters) continue;
        } else if (cs > 8) {
            break;
        }
        best = cs;
        best_chunks = chunks;
    }
    std::lock_guard<std::mutex> lk(mu);
    memo[key] = best;
    return best;
}

size_t tcs_scratch_bytes(const TcImage &img, const AnnealArgs &a) {
    const int64_t Tb = 128 / a.R;
    const int64_t groups = (int64_t(a.trials) + Tb - 1) / Tb;
    const int64_t cols = int64_t(a.trials) * a.R;
    const int L = a.delay + 2;
    return tcs::up256(size_t(groups) * L * img.KB * tcs::kABytes) + tcs::up256(size_t(cols) * a.Np) +
           tcs::up256(size_t(cols) * 16) + tcs::up256(size_t(cols) * 8) + tcs::up256(sizeof(int));
}

int tcs_anneal(const TcImage &img, const DeviceCopy &dc, const AnnealArgs &a, void *scratch, void *stream) {
    using namespace tcs;
    std::string why;
    if (!tcs_supported(img, a, &why)) return fail(SSQA_ERR_UNSUPPORTED, "streamed tensor path: " + why);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SParams p;
    std::memset(&p, 0, sizeof(p));
    p.a = a;
    p.B = dc.tcs_b;
    p.hf = dc.tcs_hf;
    p.N16 = img.N16;
    p.KB = img.KB;
    p.NCH = img.NCH;
    p.last_rows = img.N16 - 256 * (img.NCH - 1);
    p.L = a.delay + 2;
    p.Tb = 128 / a.R;
    p.jm = img.jm;
    p.NR2 = 0;
    {
        const __half2 h = __floats2half2_rn(float(a.n_rnd), float(a.n_rnd));
        std::memcpy(&p.NR2, &h, 4);
        const __half2 j = __floats2half2_rn(float(img.jm), float(img.jm));
        std::memcpy(&p.JM2, &j, 4);
    }
    p.bias = 1152.f;
    p.wait_clocks = wait_limit_clocks();
    p.i0_levels = 1;
    p.i0_mult = 2;
    p.i0_tau = 1 << 30;
    if (a.i0_max > a.I0) {
        for (int64_t v = a.I0; v < a.i0_max; v *= a.i0_mult) ++p.i0_levels;
        p.i0_mult = a.i0_mult;
        p.i0_tau = a.i0_tau;
    }
    const int64_t groups = (int64_t(a.trials) + p.Tb - 1) / p.Tb;
    const int64_t cols = int64_t(a.trials) * a.R;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // Two column groups per CTA cut the operand bytes per MAC by a third, but
    // leave a chunk's epilogue unhidden: it pays off for long chunks (SK
    // N = 8192, 256 K-blocks: 1.5x) and not for short ones (N = 2500, 80
    // K-blocks: 6 % slower).
    p.dual = img.KB >= 160 ? 1 : 0;
    const int64_t pairs = p.dual ? (groups + 1) / 2 : groups;  // CTAs per cluster rank
    int CS = tcs_cluster_size(img, a, nsm);
    uint8_t *q = static_cast<uint8_t *>(scratch);
    p.A = q;
    q += up256(size_t(groups) * p.L * p.KB * kABytes);
    p.IsB = q;
    q += up256(size_t(cols) * a.Np);
    p.eacc = reinterpret_cast<unsigned long long *>(q);
    q += up256(size_t(cols) * 16);
    p.efin = a.e_final;
    p.ebest = a.e_best;
    p.bcyc = a.best_cycle;
    q += up256(size_t(cols) * 8);
    p.err = reinterpret_cast<int *>(q);
    uint8_t *aw = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&aw), 16, st);
    if (e) return fail(SSQA_ERR_OOM, std::string("streamed tensor path: ") + cudaGetErrorString(e));
    if (img.nh) cudaMemcpyAsync(aw, img.a_w.data(), img.nh, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(p.err, 0, sizeof(int), st);
    tcs_init_kernel<<<2048, 256, 0, st>>>(p, aw, img.nh);
    if (a.init_mode == SSQA_INIT_FROM_STATE) {
        int herr = 0;
        e = cudaMemcpyAsync(&herr, p.err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (!e && herr == 2) {
            cudaFreeAsync(aw, st);
            return fail(SSQA_ERR_UNSUPPORTED, "streamed tensor path: resumed counters outside -128..127");
        }
    }
    const LaunchCfg lc = launch_cfg(p.dual != 0, a.track_best);
    void (*fn)(SParams) = lc.fn;
    const int threads = lc.threads, smem = lc.smem;
    configure_once(fn, smem);
    cudaLaunchConfig_t cfg{};
    cfg.blockDim = dim3(unsigned(threads), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the largest cluster (<= CS) that the device can place at least once
    for (; CS > 1; --CS) {
        int nclus = 0;
        cfg.gridDim = dim3(unsigned(pairs * CS), 1, 1);
        attr[0].val.clusterDim.x = unsigned(CS);
        if (cudaOccupancyMaxActiveClusters(&nclus, fn, &cfg) == cudaSuccess && nclus > 0) break;
        cudaGetLastError();
    }
    p.CS = CS;
    cfg.gridDim = dim3(unsigned(pairs * CS), 1, 1);
    attr[0].val.clusterDim.x = unsigned(CS);
    if (!e) e = cudaLaunchKernelEx(&cfg, fn, p);
    if (!e) {
        tcs_finish_kernel<<<2048, 256, 0, st>>>(p, int64_t(a.start_cycle) + a.cycles);
        e = cudaGetLastError();
    }
    int herr = 0;
    if (!e) e = cudaMemcpyAsync(&herr, p.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    cudaFreeAsync(aw, st);
    if (e) return fail(SSQA_ERR_DEVICE, std::string("streamed tensor path kernel: ") + cudaGetErrorString(e));
    if (herr) return fail(SSQA_ERR_TIMEOUT, "streamed tensor path: a bounded wait timed out");
    return SSQA_OK;
}

}  // namespace ssqa
