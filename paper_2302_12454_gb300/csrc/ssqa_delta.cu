// Delta-field path of SSQA (SSQA_ALGO_DELTA), CUDA cores.
//
// The field F_{i,c}(t) = sum_j J_ij sigma_{j,c}(t) of Eq. 6a is kept in device
// memory for every spin column.  Each cycle:
//   1. update: Eq. 6a-6c from F(t) (local field, counter, sign), exactly as
//      the other paths; every spin whose sign changed is appended to its
//      column's flip list and counted;
//   2. apply: F(t+1) = F(t) + sum_{j flipped} 2 sigma_j(t+1) J_{:,j} when the
//      cycle's flip count is small, or a dense recompute J sigma(t+1) when it
//      is large (the first tau cycles of each iteration, where J_perp = 0,
//      flip about half the spins every cycle).  The choice is taken on the
//      device from the count, so the host never waits inside the loop.
// J is symmetric, so the column J_{:,j} is row j, read contiguously.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "philox.cuh"
#include "ssqa_internal.h"

namespace ssqa {
namespace {

constexpr int kSp = 32;      // spins per block (one per lane)
constexpr int kWarps = 8;    // warps per block
constexpr int kCPB = 32;     // columns per block (four per warp)
constexpr int kKT = 128;     // bytes of K staged per dense step

struct DeltaState {
    int8_t *ring;      // [L][cols][Np] spin history
    int32_t *F;        // [cols][N]   J sigma(t)
    int32_t *list;     // [cols][N]   flipped spin indices of the last update
    int32_t *cnt;      // [2][cols]   flip counts (double buffered by cycle parity)
    unsigned long long *total;  // [2] flips of the cycle, all columns
    int64_t *e2acc;    // [cols]
    int64_t *efin;     // [cols]
    int32_t L;
    int64_t cols;
};

__host__ __device__ inline int64_t slot_of(int64_t t, int32_t L) { return ((t % L) + L) % L; }

// Eq. 6a-6c for all (column, spin) from the stored field; records flips.
template <bool kTrack>
__global__ void __launch_bounds__(kSp * kWarps) delta_update_kernel(AnnealArgs a, DeltaState s, uint32_t t, int32_t jp,
                                                                    int32_t I0, const int8_t *cur, const int8_t *old,
                                                                    int8_t *nxt,
                                                                    int32_t *cnt_w, unsigned long long *total_w) {
    constexpr int kCPW = kCPB / kWarps;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t i = int32_t(blockIdx.y) * kSp + lane;
    const int64_t cb = int64_t(blockIdx.x) * kCPB;
    const int Np = a.Np;
    uint32_t myw = 0;
    {
        const int64_t c = cb + w * kCPW + lane;
        if (lane < kCPW && c < s.cols) {
            const int32_t k = int32_t(c % a.R);
            myw = noise_word(a.seed, uint32_t(blockIdx.y) * kSp, uint32_t(k), a.trial_offset + uint32_t(c / a.R), t);
        }
    }
    unsigned flips = 0;
#pragma unroll
    for (int cc = 0; cc < kCPW; ++cc) {
        const int64_t c = cb + w * kCPW + cc;
        const uint32_t nw = __shfl_sync(0xFFFFFFFFu, myw, cc);
        const bool valid = i < a.N && c < s.cols;
        int64_t e2 = 0;
        if (valid) {
            const int32_t k = int32_t(c % a.R);
            const int64_t base = c - k;
            const int64_t r = ((nw >> spin_bit_pos(uint32_t(i))) & 1u) ? -1 : 1;
            int64_t cpl = old[(base + (k + 1 == a.R ? 0 : k + 1)) * Np + i];
            if (a.both) cpl += old[(base + (k == 0 ? a.R - 1 : k - 1)) * Np + i];
            const int64_t Fi = s.F[c * a.N + i];
            const int64_t hi = a.h[i];
            // Eq. 6a-6c
            const int64_t I = hi + Fi + int64_t(a.n_rnd) * r + int64_t(jp) * cpl;
            const int64_t v = int64_t(a.Is[c * a.N + i]) + I;
            const int32_t is_new = v >= I0 ? I0 - a.alpha : (v < -I0 ? -I0 : int32_t(v));
            a.Is[c * a.N + i] = is_new;
            const int8_t s_old = cur[c * Np + i];
            const int8_t s_new = is_new >= 0 ? 1 : -1;
            nxt[c * Np + i] = s_new;
            if (s_new != s_old) {
                // entry: spin index, sign bit set when the spin became -1
                const int32_t idx = atomicAdd(&cnt_w[c], 1);
                s.list[c * a.N + idx] = s_new > 0 ? i : int32_t(uint32_t(i) | 0x80000000u);
                ++flips;
            }
            if (kTrack) e2 = -int64_t(s_old) * (2 * hi + Fi);
        }
        if (kTrack) {
#pragma unroll
            for (int o = 16; o; o >>= 1) e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, o);
            if (lane == 0 && c < s.cols)
                atomicAdd(reinterpret_cast<unsigned long long *>(&s.e2acc[c]), static_cast<unsigned long long>(e2));
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) flips += __shfl_xor_sync(0xFFFFFFFFu, flips, o);
    if (lane == 0 && flips) atomicAdd(total_w, static_cast<unsigned long long>(flips));
}

// F(t+1) from F(t): sparse flip updates, or a dense recompute when the
// cycle's flips exceed `dense_at` (decided per launch from the device count).
__global__ void __launch_bounds__(kSp * kWarps) delta_apply_kernel(AnnealArgs a, DeltaState s, const int8_t *nxt,
                                                                   const int32_t *cnt_r, int32_t *cnt_clear,
                                                                   const unsigned long long *total_r,
                                                                   unsigned long long *total_clear,
                                                                   unsigned long long dense_at) {
    constexpr int kCPW = kCPB / kWarps;
    __shared__ uint32_t sJ[kSp][kKT / 4 + 1];
    __shared__ __align__(16) uint32_t sS[kCPB][kKT / 4];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int32_t i = int32_t(blockIdx.y) * kSp + lane;
    const int64_t cb = int64_t(blockIdx.x) * kCPB;
    const int Np = a.Np;
    // counters of the next update start at zero (other parity buffer)
    if (blockIdx.y == 0 && tid < kCPB && cb + tid < s.cols) cnt_clear[cb + tid] = 0;
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) *total_clear = 0;
    const bool dense = *total_r >= dense_at;
    if (dense) {
        int32_t F[kCPW];
#pragma unroll
        for (int cc = 0; cc < kCPW; ++cc) F[cc] = 0;
        for (int32_t k0 = 0; k0 < Np; k0 += kKT) {
            {
                const int32_t row = int32_t(blockIdx.y) * kSp + tid / 8;
                const int32_t kk = k0 + (tid % 8) * 16;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (row < a.N && kk < Np) v = *reinterpret_cast<const uint4 *>(a.J_pad + int64_t(row) * Np + kk);
                uint32_t *d = &sJ[tid / 8][(tid % 8) * 4];
                d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
            }
            {
                const int64_t col = cb + tid / 8;
                const int32_t kk = k0 + (tid % 8) * 16;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (col < s.cols && kk < Np) v = *reinterpret_cast<const uint4 *>(nxt + col * Np + kk);
                *reinterpret_cast<uint4 *>(&sS[tid / 8][(tid % 8) * 4]) = v;
            }
            __syncthreads();
#pragma unroll 8
            for (int q = 0; q < kKT / 4; ++q) {
                const int jw = int(sJ[lane][q]);
#pragma unroll
                for (int cc = 0; cc < kCPW; ++cc) F[cc] = __dp4a(jw, int(sS[w * kCPW + cc][q]), F[cc]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int cc = 0; cc < kCPW; ++cc) {
            const int64_t c = cb + w * kCPW + cc;
            if (i < a.N && c < s.cols) s.F[c * a.N + i] = F[cc];
        }
        return;
    }
#pragma unroll
    for (int cc = 0; cc < kCPW; ++cc) {
        const int64_t c = cb + w * kCPW + cc;
        if (c >= s.cols || i >= a.N) continue;
        const int32_t n = cnt_r[c];
        if (n == 0) continue;
        const int32_t *lst = s.list + c * a.N;
        const int8_t *Jc = a.J_pad + i;
        // sigma_j went from -s to s: F_i += 2 s J_ij  (J_ij = J_ji, row j)
        int32_t d0 = 0, d1 = 0;
        int32_t q = 0;
        for (; q + 1 < n; q += 2) {
            const uint32_t e0 = uint32_t(lst[q]), e1 = uint32_t(lst[q + 1]);
            const int32_t v0 = Jc[int64_t(e0 & 0x7FFFFFFFu) * Np];
            const int32_t v1 = Jc[int64_t(e1 & 0x7FFFFFFFu) * Np];
            d0 += (e0 >> 31) ? -v0 : v0;
            d1 += (e1 >> 31) ? -v1 : v1;
        }
        if (q < n) {
            const uint32_t e0 = uint32_t(lst[q]);
            const int32_t v0 = Jc[int64_t(e0 & 0x7FFFFFFFu) * Np];
            d0 += (e0 >> 31) ? -v0 : v0;
        }
        s.F[c * a.N + i] += 2 * (d0 + d1);
    }
}

__global__ void delta_init_kernel(AnnealArgs a, DeltaState s) {
    const int64_t cols = s.cols;
    const int64_t n = cols * a.Np;
    const int64_t t0 = a.start_cycle;
    for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = x / a.Np;
        const int32_t i = int32_t(x % a.Np);
        if (i >= a.N) {
            for (int l = 0; l < s.L; ++l) s.ring[(l * cols + c) * a.Np + i] = 0;
            continue;
        }
        const int32_t k = int32_t(c % a.R);
        const int64_t trial = c / a.R;
        int8_t s0;
        if (a.init_mode == SSQA_INIT_FROM_STATE) {
            s0 = a.sigma[c * a.N + i];
        } else {
            if (a.init_mode == SSQA_INIT_RANDOM) {
                const uint32_t w = noise_word(a.seed, uint32_t(i), uint32_t(k), a.trial_offset + uint32_t(trial),
                                              0xFFFFFFFFu);
                s0 = ((w >> spin_bit_pos(uint32_t(i))) & 1u) ? int8_t(-1) : int8_t(1);
            } else {
                s0 = -1;
            }
            a.Is[c * a.N + i] = 0;
        }
        s.ring[(slot_of(t0, s.L) * cols + c) * a.Np + i] = s0;
        for (int l = 1; l <= a.delay; ++l) {
            int8_t v = s0;
            if (a.init_mode == SSQA_INIT_FROM_STATE)
                v = a.hist[((trial * a.delay + (l - 1)) * a.R + k) * int64_t(a.N) + i];
            s.ring[(slot_of(t0 - l, s.L) * cols + c) * a.Np + i] = v;
        }
    }
    if (blockIdx.x == 0)
        for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) {
            s.e2acc[c] = 0;
            s.cnt[c] = 0;
            s.cnt[cols + c] = 0;
            if (a.track_best) {
                a.e_best[c] = LLONG_MAX;
                a.best_cycle[c] = -1;
            }
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.total[0] = ~0ull;  // the first apply recomputes F densely
        s.total[1] = 0;
    }
}

// E_best / best_cycle update with the energies of sigma(tc); the row of the
// energy trace for tc, when traced.
__global__ void delta_best_kernel(int64_t *src, int halve, int64_t *e_best, int32_t *best_cycle, int64_t cols,
                                  int32_t tc, int64_t *trace_row) {
    for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < cols; c += int64_t(gridDim.x) * blockDim.x) {
        int64_t E = src[c];
        if (halve) {
            E /= 2;
            src[c] = 0;
        }
        if (trace_row) trace_row[c] = E;
        if (E < e_best[c]) {
            e_best[c] = E;
            best_cycle[c] = tc;
        }
    }
}

__global__ void delta_finish_kernel(AnnealArgs a, DeltaState s, int64_t tf) {
    const int64_t cols = s.cols;
    const int64_t n = cols * a.N;
    for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = x / a.N;
        const int32_t i = int32_t(x % a.N);
        a.sigma[x] = s.ring[(slot_of(tf, s.L) * cols + c) * a.Np + i];
        if (a.hist) {
            const int32_t k = int32_t(c % a.R);
            const int64_t trial = c / a.R;
            for (int l = 0; l < a.delay; ++l)
                a.hist[((trial * a.delay + l) * a.R + k) * int64_t(a.N) + i] =
                    s.ring[(slot_of(tf - 1 - l, s.L) * cols + c) * a.Np + i];
        }
    }
}

inline int launch_check(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SSQA_ERR_DEVICE, std::string(what) + ": " + cudaGetErrorString(e));
    return SSQA_OK;
}

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Probe flip lists: every column lists spins 0..m-1 as flipped.
__global__ void delta_probe_kernel(DeltaState s, int32_t N, int32_t m, int32_t *cnt) {
    for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < s.cols * int64_t(m);
         x += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = x / m;
        const int32_t q = int32_t(x % m);
        s.list[c * N + q] = q;
        if (q == 0) cnt[c] = m;
    }
}

// Autotuned dense/sparse switch: on the first anneal of a shape (N, columns)
// one dense pass and one sparse pass with N/16 flips per column are timed
// with CUDA events on the launching stream; the cycle then goes dense once
// its total flips cost more, by that measurement, than a dense pass.
unsigned long long dense_threshold(const AnnealArgs &a, const DeltaState &s, dim3 grid, cudaStream_t st) {
    static std::mutex mu;
    static std::map<std::pair<int64_t, int64_t>, unsigned long long> cache;
    const auto key = std::make_pair(int64_t(a.N), s.cols);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    unsigned long long thr = (unsigned long long)(s.cols) * (unsigned long long)(a.N) / 4ull + 1ull;
    const int32_t m = a.N >= 16 ? a.N / 16 : 1;
    cudaEvent_t e0, e1, e2, e3;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1) || cudaEventCreate(&e2) || cudaEventCreate(&e3)) {
        cudaGetLastError();
        return thr;
    }
    int8_t *spins = s.ring;  // any spin slot: the probes only read it
    unsigned long long *tot = s.total;
    const unsigned long long dense_now = 0ull, never = ~0ull;
    cudaMemsetAsync(s.F, 0, size_t(s.cols) * size_t(a.N) * 4, st);
    cudaMemsetAsync(spins, 0, size_t(s.cols) * size_t(a.Np), st);
    cudaMemsetAsync(tot, 0, 16, st);
    delta_probe_kernel<<<1024, 256, 0, st>>>(s, a.N, m, s.cnt);
    cudaEventRecord(e0, st);
    delta_apply_kernel<<<grid, kSp * kWarps, 0, st>>>(a, s, spins, s.cnt, s.cnt + s.cols, tot, tot + 1, dense_now);
    cudaEventRecord(e1, st);
    delta_probe_kernel<<<1024, 256, 0, st>>>(s, a.N, m, s.cnt);
    cudaEventRecord(e2, st);
    delta_apply_kernel<<<grid, kSp * kWarps, 0, st>>>(a, s, spins, s.cnt, s.cnt + s.cols, tot, tot + 1, never);
    cudaEventRecord(e3, st);
    float t_dense = 0.f, t_sparse = 0.f;
    if (cudaEventSynchronize(e3) == cudaSuccess && cudaEventElapsedTime(&t_dense, e0, e1) == cudaSuccess &&
        cudaEventElapsedTime(&t_sparse, e2, e3) == cudaSuccess && t_sparse > 0.f) {
        const double per_flip = double(t_sparse) / (double(s.cols) * m);
        thr = (unsigned long long)(double(t_dense) / per_flip) + 1ull;
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    cudaEventDestroy(e3);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = thr;
    return thr;
}

}  // namespace

size_t delta_scratch_bytes(const AnnealArgs &a) {
    const size_t cols = size_t(a.trials) * a.R;
    return up256(size_t(a.delay + 2) * cols * size_t(a.Np)) + 2 * up256(cols * size_t(a.N) * 4) +
           up256(2 * cols * 4) + up256(16) + 2 * up256(cols * 8);
}

int delta_anneal(const AnnealArgs &a, void *scratch, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DeltaState s;
    s.cols = int64_t(a.trials) * a.R;
    s.L = a.delay + 2;
    uint8_t *p = static_cast<uint8_t *>(scratch);
    s.ring = reinterpret_cast<int8_t *>(p);
    p += up256(size_t(s.L) * size_t(s.cols) * size_t(a.Np));
    s.F = reinterpret_cast<int32_t *>(p);
    p += up256(size_t(s.cols) * size_t(a.N) * 4);
    s.list = reinterpret_cast<int32_t *>(p);
    p += up256(size_t(s.cols) * size_t(a.N) * 4);
    s.cnt = reinterpret_cast<int32_t *>(p);
    p += up256(2 * size_t(s.cols) * 4);
    s.total = reinterpret_cast<unsigned long long *>(p);
    p += up256(16);
    s.e2acc = reinterpret_cast<int64_t *>(p);
    p += up256(size_t(s.cols) * 8);
    s.efin = a.e_final ? a.e_final : reinterpret_cast<int64_t *>(p);
    const int64_t t0 = a.start_cycle;
    const int64_t gx = (s.cols + kCPB - 1) / kCPB, gy = (a.N + kSp - 1) / kSp;
    if (gx > INT32_MAX || gy > 65535) return fail(SSQA_ERR_UNSUPPORTED, "delta path: problem exceeds the grid");
    const dim3 grid{unsigned(gx), unsigned(gy), 1u};
    const unsigned long long dense_at = dense_threshold(a, s, grid, st);
    delta_init_kernel<<<1024, 256, 0, st>>>(a, s);
    if (int rc = launch_check("delta init")) return rc;
    // F(t0) = J sigma(t0): dense (total[0] starts saturated)
    delta_apply_kernel<<<grid, kSp * kWarps, 0, st>>>(a, s, s.ring + slot_of(t0, s.L) * s.cols * a.Np, s.cnt,
                                                       s.cnt + s.cols, s.total, s.total + 1, dense_at);
    if (int rc = launch_check("delta apply")) return rc;
    const int64_t period = int64_t(a.tau) * (a.beta + 1);
    for (int64_t c = 0; c < a.cycles; ++c) {
        const int64_t t = t0 + c;
        const int par = int(c & 1);  // update writes cnt/total[1 - par]... see below
        const int32_t jp = a.jperp_min + int32_t((t % period) / a.tau) * a.jperp_step;
        const int32_t I0 = i0_at(a, t);
        const int8_t *cur = s.ring + slot_of(t, s.L) * s.cols * a.Np;
        const int8_t *old = s.ring + slot_of(t - a.delay, s.L) * s.cols * a.Np;
        int8_t *nxt = s.ring + slot_of(t + 1, s.L) * s.cols * a.Np;
        // buffers: the update of cycle c writes parity w = (c + 1) & 1 (the
        // initial dense apply cleared it), the apply reads it and clears 1 - w
        const int wp = (par + 1) & 1;
        int32_t *cnt_w = s.cnt + wp * s.cols;
        int32_t *cnt_o = s.cnt + (1 - wp) * s.cols;
        if (a.track_best && c > 0) {
            delta_update_kernel<true><<<grid, kSp * kWarps, 0, st>>>(a, s, uint32_t(t), jp, I0, cur, old, nxt, cnt_w,
                                                                     s.total + wp);
            delta_best_kernel<<<256, 256, 0, st>>>(s.e2acc, 1, a.e_best, a.best_cycle, s.cols, int32_t(t),
                                                   a.e_trace ? a.e_trace + (c - 1) * s.cols : nullptr);
        } else {
            delta_update_kernel<false><<<grid, kSp * kWarps, 0, st>>>(a, s, uint32_t(t), jp, I0, cur, old, nxt, cnt_w,
                                                                      s.total + wp);
        }
        if (int rc = launch_check("delta update")) return rc;
        delta_apply_kernel<<<grid, kSp * kWarps, 0, st>>>(a, s, nxt, cnt_w, cnt_o, s.total + wp, s.total + (1 - wp),
                                                           dense_at);
        if (int rc = launch_check("delta apply")) return rc;
    }
    const int64_t tf = t0 + a.cycles;
    delta_finish_kernel<<<1024, 256, 0, st>>>(a, s, tf);
    if (int rc = launch_check("delta finish")) return rc;
    if (a.e_final || a.track_best) {
        if (int rc = energy_launch(a.J_pad, a.Np, a.h, a.N, s.ring + slot_of(tf, s.L) * s.cols * a.Np, a.Np, s.cols,
                                   s.efin, stream))
            return rc;
        if (a.track_best && a.cycles > 0) {
            delta_best_kernel<<<256, 256, 0, st>>>(s.efin, 0, a.e_best, a.best_cycle, s.cols, int32_t(tf),
                                                   a.e_trace ? a.e_trace + (a.cycles - 1) * s.cols : nullptr);
            if (int rc = launch_check("delta best")) return rc;
        }
    }
    return SSQA_OK;
}

}  // namespace ssqa
