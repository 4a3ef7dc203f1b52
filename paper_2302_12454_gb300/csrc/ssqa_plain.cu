// Plain CUDA-core path of SSQA and the energy kernel.
//
// One kernel launch per annealing cycle (Eq. 6a-6c of the paper), every
// spin of every replica and trial updated in parallel (Sec. 3.2: "all the
// N*R spin states are updated in parallel").  The field product
// sum_j J_ij sigma_{j,k}(t) is an int8 dot product (dp4a) over J rows and
// spin columns staged in shared memory; the local field, counter and sign
// follow in the same thread.  This is the straightforward GPU port against
// which the persistent tensor-core path is measured.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "philox.cuh"
#include "ssqa_internal.h"

namespace ssqa {
namespace {

constexpr int kSpins = 32;          // spins per block (one per lane)
constexpr int kCols = 8;            // warps per block
constexpr int kColsPerBlock = 32;   // spin columns per block (four per warp)
constexpr int kKT = 128;            // bytes of K staged per step

struct PlainState {
    int8_t *ring;     // [L][cols][Np] spin history, slot(t) = t mod L
    int64_t *e2acc;   // [cols] twice the energy of the current state
    int64_t *efin;    // [cols] final energy (scratch when e_final is null)
    int32_t L;
    int64_t cols;
};

__host__ __device__ inline int64_t slot_of(int64_t t, int32_t L) { return ((t % L) + L) % L; }

__global__ void plain_init_kernel(AnnealArgs a, PlainState s) {
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
            if (a.track_best) {
                a.e_best[c] = LLONG_MAX;
                a.best_cycle[c] = -1;
            }
        }
}

// One synchronous update t -> t+1 of all (column c, spin i).  A block owns
// 32 spins (one per lane) and 32 columns (four per warp): each J word staged
// in shared memory feeds four dot products.  The host passes the cycle's
// J_perp value and the history slots, so the kernel does no index division.
template <bool kTrack>
__global__ void __launch_bounds__(kSpins * kCols) plain_cycle_kernel(AnnealArgs a, int64_t cols, int64_t *e2acc,
                                                                     uint32_t t, int32_t jp, int32_t I0,
                                                                     const int8_t *cur, const int8_t *old,
                                                                     int8_t *nxt) {
    constexpr int kCPW = kColsPerBlock / kCols;  // columns per warp (thread)
    __shared__ uint32_t sJ[kSpins][kKT / 4 + 1];
    __shared__ __align__(16) uint32_t sS[kColsPerBlock][kKT / 4];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int32_t i = int32_t(blockIdx.y) * kSpins + lane;
    const int64_t cb = int64_t(blockIdx.x) * kColsPerBlock;
    const int Np = a.Np;

    int32_t F[kCPW];
#pragma unroll
    for (int cc = 0; cc < kCPW; ++cc) F[cc] = 0;
    for (int32_t k0 = 0; k0 < Np; k0 += kKT) {
        {
            const int32_t row = int32_t(blockIdx.y) * kSpins + tid / 8;
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
            if (col < cols && kk < Np) v = *reinterpret_cast<const uint4 *>(cur + col * Np + kk);
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

    // noise words: lane cc computes the Philox call of column cc of this warp
    uint32_t myw = 0;
    {
        const int64_t c = cb + w * kCPW + lane;
        if (lane < kCPW && c < cols) {
            const int32_t k = int32_t(c % a.R);
            const uint32_t trial = a.trial_offset + uint32_t(c / a.R);
            myw = noise_word(a.seed, uint32_t(blockIdx.y) * kSpins, uint32_t(k), trial, t);
        }
    }
#pragma unroll
    for (int cc = 0; cc < kCPW; ++cc) {
        const int64_t c = cb + w * kCPW + cc;
        const uint32_t nw = __shfl_sync(0xFFFFFFFFu, myw, cc);
        const bool valid = i < a.N && c < cols;
        int64_t e2 = 0;
        if (valid) {
            const int32_t k = int32_t(c % a.R);
            const int64_t base = c - k;  // column of replica 0 of this trial
            const int64_t r = ((nw >> spin_bit_pos(uint32_t(i))) & 1u) ? -1 : 1;
            // Eq. 6a: h + J sigma(t) + n_rnd r + J_perp(t) sigma_{k+1}(t - d)
            int64_t cpl = old[(base + (k + 1 == a.R ? 0 : k + 1)) * Np + i];
            if (a.both) cpl += old[(base + (k == 0 ? a.R - 1 : k - 1)) * Np + i];
            const int64_t hi = a.h[i];
            const int64_t I = hi + F[cc] + int64_t(a.n_rnd) * r + int64_t(jp) * cpl;
            // Eq. 6b: saturating integral counter
            const int64_t v = int64_t(a.Is[c * a.N + i]) + I;
            const int32_t is_new = v >= I0 ? I0 - a.alpha : (v < -I0 ? -I0 : int32_t(v));
            a.Is[c * a.N + i] = is_new;
            // Eq. 6c
            nxt[c * Np + i] = is_new >= 0 ? 1 : -1;
            if (kTrack) e2 = -int64_t(cur[c * Np + i]) * (2 * hi + F[cc]);  // 2 E of sigma(t), Eq. 5
        }
        if (kTrack) {
#pragma unroll
            for (int o = 16; o; o >>= 1) e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, o);
            if (lane == 0 && c < cols)
                atomicAdd(reinterpret_cast<unsigned long long *>(&e2acc[c]), static_cast<unsigned long long>(e2));
        }
    }
}

// e_best / best_cycle update with the energy of the state at cycle tc.
// E_best / best_cycle update with the energies of sigma(tc); the row of the
// energy trace for tc, when traced.
__global__ void plain_best_kernel(int64_t *src, int halve, int64_t *e_best, int32_t *best_cycle, int64_t cols,
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

__global__ void plain_finish_kernel(AnnealArgs a, PlainState s, int64_t tf) {
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

// E' = -sum_i s_i (h_i + F_i / 2), F = J s; each block handles kV vectors,
// one warp per J row at a time, lanes striding over the row (coalesced).
constexpr int kV = 8;

__global__ void __launch_bounds__(256) energy_kernel(const int8_t *J_pad, int32_t Np, const int32_t *h, int32_t N,
                                                     const int8_t *sigma, int64_t pitch, int64_t count, int64_t *E) {
    extern __shared__ __align__(16) uint8_t sm[];
    int8_t *sv = reinterpret_cast<int8_t *>(sm);  // [kV][Np]
    __shared__ long long red[kV][8];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t r0 = int64_t(blockIdx.x) * kV;
    const int nv = int(count - r0 < kV ? count - r0 : kV);
    for (int x = tid; x < kV * Np; x += blockDim.x) {
        const int v = x / Np, j = x % Np;
        sv[x] = (v < nv && j < N) ? sigma[(r0 + v) * pitch + j] : int8_t(0);
    }
    __syncthreads();
    long long e2[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) e2[v] = 0;
    for (int32_t i = w; i < N; i += 8) {
        int F[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) F[v] = 0;
        const uint32_t *row = reinterpret_cast<const uint32_t *>(J_pad + int64_t(i) * Np);
        for (int32_t q = lane; q < Np / 4; q += 32) {
            const int jw = int(row[q]);
#pragma unroll
            for (int v = 0; v < kV; ++v) F[v] = __dp4a(jw, reinterpret_cast<const int *>(sv + v * Np)[q], F[v]);
        }
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            int f = F[v];
#pragma unroll
            for (int o = 16; o; o >>= 1) f += __shfl_xor_sync(0xFFFFFFFFu, f, o);
            if (lane == 0) e2[v] -= (long long)sv[v * Np + i] * (2LL * h[i] + f);
        }
    }
    if (lane == 0)
        for (int v = 0; v < kV; ++v) red[v][w] = e2[v];
    __syncthreads();
    if (tid < nv) {
        long long s = 0;
        for (int q = 0; q < 8; ++q) s += red[tid][q];
        E[r0 + tid] = s / 2;
    }
}

inline int launch_check(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SSQA_ERR_DEVICE, std::string(what) + ": " + cudaGetErrorString(e));
    return SSQA_OK;
}

}  // namespace

size_t plain_scratch_bytes(const AnnealArgs &a) {
    const size_t cols = size_t(a.trials) * a.R;
    const size_t ring = size_t(a.delay + 2) * cols * size_t(a.Np);
    return (ring + 255) / 256 * 256 + 2 * cols * 8 + 256;
}

int energy_launch(const int8_t *J_pad, int32_t Np, const int32_t *h, int32_t N, const int8_t *sigma, int64_t pitch,
                  int64_t count, int64_t *E, void *stream) {
    if (count <= 0) return SSQA_OK;
    const size_t smem = size_t(kV) * Np;
    if (smem > 200 * 1024) return fail(SSQA_ERR_UNSUPPORTED, "energy: N too large for one block's shared memory");
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    const int64_t blocks = (count + kV - 1) / kV;
    if (blocks > INT32_MAX) return fail(SSQA_ERR_INVALID_ARG, "energy: too many vectors");
    energy_kernel<<<unsigned(blocks), 256, smem, static_cast<cudaStream_t>(stream)>>>(J_pad, Np, h, N, sigma, pitch,
                                                                                       count, E);
    return launch_check("energy kernel");
}

int plain_anneal(const AnnealArgs &a, void *scratch, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PlainState s;
    s.cols = int64_t(a.trials) * a.R;
    s.L = a.delay + 2;
    const size_t ring = size_t(s.L) * size_t(s.cols) * size_t(a.Np);
    uint8_t *base = static_cast<uint8_t *>(scratch);
    s.ring = reinterpret_cast<int8_t *>(base);
    s.e2acc = reinterpret_cast<int64_t *>(base + (ring + 255) / 256 * 256);
    s.efin = a.e_final ? a.e_final : s.e2acc + s.cols;
    const int64_t t0 = a.start_cycle;
    plain_init_kernel<<<1024, 256, 0, st>>>(a, s);
    if (int rc = launch_check("plain init")) return rc;
    const int64_t gx = (s.cols + kColsPerBlock - 1) / kColsPerBlock;
    const int64_t gy = (a.N + kSpins - 1) / kSpins;
    if (gx > INT32_MAX || gy > 65535) return fail(SSQA_ERR_UNSUPPORTED, "plain path: problem exceeds the grid");
    const dim3 grid{unsigned(gx), unsigned(gy), 1u};
    const int64_t period = int64_t(a.tau) * (a.beta + 1);
    for (int64_t c = 0; c < a.cycles; ++c) {
        const int64_t t = t0 + c;
        const int32_t jp = a.jperp_min + int32_t((t % period) / a.tau) * a.jperp_step;  // Table 2 schedule
        const int32_t I0 = i0_at(a, t);
        const int8_t *cur = s.ring + slot_of(t, s.L) * s.cols * a.Np;
        const int8_t *old = s.ring + slot_of(t - a.delay, s.L) * s.cols * a.Np;
        int8_t *nxt = s.ring + slot_of(t + 1, s.L) * s.cols * a.Np;
        if (a.track_best && c > 0) {
            plain_cycle_kernel<true><<<grid, kSpins * kCols, 0, st>>>(a, s.cols, s.e2acc, uint32_t(t), jp, I0, cur,
                                                                       old, nxt);
            plain_best_kernel<<<256, 256, 0, st>>>(s.e2acc, 1, a.e_best, a.best_cycle, s.cols, int32_t(t),
                                                   a.e_trace ? a.e_trace + (c - 1) * s.cols : nullptr);
        } else {
            plain_cycle_kernel<false><<<grid, kSpins * kCols, 0, st>>>(a, s.cols, s.e2acc, uint32_t(t), jp, I0, cur,
                                                                        old, nxt);
        }
        if (int rc = launch_check("plain cycle")) return rc;
    }
    const int64_t tf = t0 + a.cycles;
    plain_finish_kernel<<<1024, 256, 0, st>>>(a, s, tf);
    if (int rc = launch_check("plain finish")) return rc;
    if (a.e_final || a.track_best) {
        if (int rc = energy_launch(a.J_pad, a.Np, a.h, a.N, s.ring + slot_of(tf, s.L) * s.cols * a.Np, a.Np, s.cols,
                                   s.efin, stream))
            return rc;
        if (a.track_best && a.cycles > 0) {
            plain_best_kernel<<<256, 256, 0, st>>>(s.efin, 0, a.e_best, a.best_cycle, s.cols, int32_t(tf),
                                                   a.e_trace ? a.e_trace + (a.cycles - 1) * s.cols : nullptr);
            if (int rc = launch_check("plain best")) return rc;
        }
    }
    return SSQA_OK;
}

}  // namespace ssqa
