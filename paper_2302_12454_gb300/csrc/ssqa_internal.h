// Internal declarations shared by the host side (ssqa_api.cpp, ssqa_server.cpp)
// and the CUDA kernels (ssqa_plain.cu, ssqa_tc.cu) of the SSQA library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ssqa.h"

namespace ssqa {

// Record an error for ssqa_last_error() and return `code`.
int fail(int code, const std::string &msg);

// ---------------------------------------------------------------------------
// Tensor-core operand image of an instance.  The field product of Eq. 6a,
// F_{i,c} = sum_j J_ij sigma_{j,c}, runs as D = A * B^T on tcgen05 with
//   A[c][j] = sigma_{j,c}           (128 columns c = trial*R + k of one CTA)
//   B[i][j] = J_ij / jm             (spin rows i, FP8 E4M3, exact small ints)
// plus `nh` extra K columns that add h_i / jm:  A[c][N16 + m] = weight_m,
// B[i][N16 + m] = digit_m(h_i / jm), weights 1, 16, 256, 256, ...
// so D_{c,i} = (F_{i,c} + h_i) / jm exactly.  Both operands use the
// no-swizzle K-major core-matrix layout: element (r, k) at byte
//   (r / 8) * (Kp * 8) + (k / 16) * 128 + (r % 8) * 16 + (k % 16).
// ---------------------------------------------------------------------------
struct TcImage {
    bool ok = false;          // instance representable exactly on this path
    std::string why;          // reason when !ok
    int32_t jm = 1;           // common factor of J' and h'
    int32_t N16 = 0;          // N rounded up to 16
    int32_t nh = 0;           // number of h digit columns
    int32_t Kp = 0;           // K extent (multiple of 32)
    int32_t nchunk = 0;       // MMA N-chunks (<= 2): rows [0, chunk_rows[0]) then the rest
    int32_t chunk_rows[2] = {0, 0};
    int32_t Brows = 0;        // sum of chunk rows
    std::vector<uint8_t> b;   // B image, Brows * Kp bytes
    std::vector<uint8_t> a_w; // e4m3 weights of the h columns (nh bytes)
    std::vector<int32_t> h_unit; // h_i / jm (N)
    int64_t max_row_sum = 0;     // max_i (|h_i| + sum_j |J_ij|) / jm: bound of every partial sum of D
    int64_t max_h_unit = 0;      // max_i |h_i| / jm
    // Streamed image (instances too large for one SM): B in 256-spin chunks
    // and 32-wide K-blocks, block (ch, kb) of 256 x 32 bytes at
    // (ch * KB + kb) * 8192, element (r, k) at (r/8)*256 + (k/16)*128 + (r%8)*16 + k%16.
    bool s_ok = false;
    int32_t KB = 0, NCH = 0;
    std::vector<uint8_t> bs;
};

struct DeviceCopy {
    int8_t *J = nullptr;       // N*N int8
    int8_t *J_pad = nullptr;   // N rows of Np bytes (zero padded), plain path
    int32_t Np = 0;            // N rounded up to 16
    int32_t *h = nullptr;      // N int32
    uint8_t *tc_b = nullptr;   // B image
    int32_t *tc_h_unit = nullptr;
    uint8_t *tcs_b = nullptr;  // streamed B image
    float *tcs_hf = nullptr;   // h / jm as float
};

}  // namespace ssqa

struct ssqa_ising {
    int32_t N = 0;
    std::vector<int8_t> J;     // N*N
    std::vector<int32_t> h;    // N
    int64_t e_offset = 0;
    ssqa::TcImage tc;
    std::mutex mu;
    std::map<int, ssqa::DeviceCopy> dev;  // per CUDA device
};

namespace ssqa {

// Device copy of an instance on the current device (created on first use,
// from the library pool, on stream `st`, complete when this returns).
int device_copy(const ssqa_ising *ising, DeviceCopy **out, cudaStream_t st);

// ---------------------------------------------------------------------------
// Launch descriptors (device pointers only)
// ---------------------------------------------------------------------------
struct AnnealArgs {
    int32_t N, R, trials, cycles;
    int32_t I0, alpha, n_rnd;
    int32_t jperp_min, jperp_step, beta, tau;
    int32_t delay, both, init_mode, start_cycle;
    uint32_t trial_offset;
    uint64_t seed;
    int32_t i0_max, i0_mult, i0_tau;  // I0 schedule (i0_max <= I0: fixed)
    bool track_best;
    // instance
    const int8_t *J;
    const int8_t *J_pad;  // rows padded to Np bytes
    int32_t Np;
    const int32_t *h;
    // state / results (device)
    int8_t *sigma;        // [cols][N]   in (resume) / out
    int8_t *hist;         // [trials][d][R][N] in/out (may be null if d == 0)
    int32_t *Is;          // [cols][N]   in/out
    int64_t *e_final;     // [cols] or null
    int64_t *e_best;      // [cols] or null
    int64_t *e_trace;     // [cycles][cols] or null: E(sigma(t0 + c + 1)), needs track_best
    int32_t *best_cycle;  // [cols] or null
};

// Bytes of scratch the plain path needs for `a` (see plain_anneal).
size_t plain_scratch_bytes(const AnnealArgs &a);
// Plain CUDA-core path: one launch per cycle.  `scratch` must hold
// plain_scratch_bytes(a) bytes of device memory (256-byte aligned).
int plain_anneal(const AnnealArgs &a, void *scratch, void *stream);

// Delta-field path: F = J sigma kept per column, sparse flip updates or a
// dense recompute per cycle.  `scratch` holds delta_scratch_bytes(a) bytes.
size_t delta_scratch_bytes(const AnnealArgs &a);
int delta_anneal(const AnnealArgs &a, void *scratch, void *stream);

// Energy E' of `count` spin rows of `pitch` bytes (device pointers), using
// the zero-padded J rows (pitch Np).  No scratch.
int energy_launch(const int8_t *J_pad, int32_t Np, const int32_t *h, int32_t N, const int8_t *sigma,
                  int64_t pitch, int64_t count, int64_t *E, void *stream);

// Tensor-core path: whether the resident kernel can run this problem.
bool tc_supported(const TcImage &img, const AnnealArgs &a, std::string *why);
// Variant of the resident kernel for a problem it supports: byte or half2
// counters, shuffle or shared-memory replica exchange, FP16 or FP32
// accumulator.
struct TcVariant {
    bool bytes = false, shfl = false, f16 = false;
};
TcVariant tc_variant(const TcImage &img, const AnnealArgs &a);
int tc_anneal(const TcImage &img, const DeviceCopy &dc, const AnnealArgs &a, void *stream);
// Several resident-kernel problems: those of one kernel variant run in one
// launch (or a few, 48 problems at most per launch), the others alone; all on
// `stream`, complete on return.  *launches (if non-NULL) is incremented per
// kernel launch.
struct TcBatchItem {
    const TcImage *img;
    const DeviceCopy *dc;
    AnnealArgs a;
};
int tc_anneal_batch(const TcBatchItem *items, int count, int *launches, void *stream);
// Kernel variant of a resident-kernel problem that has a batched launch, as
// a small non-negative key (problems with equal keys can share a launch);
// -1 when the problem has no batched launch.
int tc_batch_key(const TcImage &img, const AnnealArgs &a);
// The same for a problem given by its instance and parameters (host only):
// -1 unless ssqa_anneal would run it on the resident kernel with a batched
// variant.
int batch_key(const ssqa_ising *ising, const ssqa_params *params);

// I0 of cycle t: fixed, or the SSA schedule of Sec. 4.4.
inline int32_t i0_at(const AnnealArgs &a, int64_t t) {
    if (a.i0_max <= a.I0) return a.I0;
    int32_t levels = 1;
    for (int64_t v = a.I0; v < a.i0_max; v *= a.i0_mult) ++levels;
    const int64_t l = (t % (int64_t(a.i0_tau) * levels)) / a.i0_tau;
    int64_t v = a.I0;
    for (int64_t q = 0; q < l; ++q) v *= a.i0_mult;
    return int32_t(v);
}

// Stream-ordered allocation from the library's own pool on the current device.
// The pool never inserts waits between streams to reuse memory (only memory
// whose free has already completed is reused), so concurrent anneals on
// different streams stay independent.
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st);

// Streamed tensor-core path (N too large for the resident kernel).
bool tcs_supported(const TcImage &img, const AnnealArgs &a, std::string *why);
size_t tcs_scratch_bytes(const TcImage &img, const AnnealArgs &a);
// CTAs per cluster of the streamed launch on a device with `nsm` SMs (the
// cluster shares one column group's, or pair of groups', 256-spin chunks).
int tcs_cluster_size(const TcImage &img, const AnnealArgs &a, int nsm);
int tcs_anneal(const TcImage &img, const DeviceCopy &dc, const AnnealArgs &a, void *scratch, void *stream);

// Bound, in SM clocks, of every wait a tensor-core kernel makes for the
// tensor cores, a copy or another warp (ssqa_set_wait_limit; default 8e9,
// about 4 s at 2 GHz).
long long wait_limit_clocks();

// Current device has compute capability 10.x (sm_100 family).
int check_device(int *device);

}  // namespace ssqa
