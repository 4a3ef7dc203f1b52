/*
 * ssqa.h -- C ABI of the GB300 (sm_103a) library for Stochastic Simulated
 * Quantum Annealing (SSQA; Onizawa, Sasaki, Shin, Gross, Hanyu, arXiv
 * 2302.12454).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an int status: SSQA_OK (0), SSQA_PENDING (> 0, only
 *    from ssqa_poll) or a negative SSQA_ERR_* code.  No call aborts, traps or
 *    exits; ssqa_last_error() gives a human-readable reason for the last
 *    failure on the calling thread.
 *  - All real-valued quantities of the paper (h, J, I0, n_rnd, J_perp, alpha,
 *    energies) are passed as integers scaled by one factor S chosen by the
 *    caller (S = 12 makes every constant of Table 2 an integer: I0' = 24,
 *    n_rnd' = 12, J_perp' in {0, 2, 4, 6}, alpha' = 1).  The dynamics of
 *    Eq. 6 are invariant under this scaling, so results are bit-exact
 *    integers.
 *  - Buffers passed in are owned by the caller and only read (inputs) or
 *    written (outputs) during the call (or, for asynchronous device-pointer
 *    calls, until the stream reaches that point).  Objects returned through
 *    `**out` are owned by the library and released by the matching *_free /
 *    *_destroy call.
 *  - Pointers are host pointers unless a call says otherwise.  With
 *    SSQA_FLAG_DEVICE_PTRS, the state and result pointers of ssqa_anneal and
 *    the sigma / energy pointers of ssqa_energy are device pointers on the
 *    current CUDA device, and the call is asynchronous on `cuda_stream`.
 *  - The compute path is CUDA only.  If no sm_100-family GPU is present, the
 *    compute calls return SSQA_ERR_DEVICE; there is no CPU fallback.
 */
#ifndef SSQA_H
#define SSQA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
#define SSQA_OK 0
#define SSQA_PENDING 1
#define SSQA_ERR_INVALID_ARG (-1)
#define SSQA_ERR_UNSUPPORTED (-2)
#define SSQA_ERR_OOM (-3)
#define SSQA_ERR_BUDGET (-4)
#define SSQA_ERR_TIMEOUT (-5)
#define SSQA_ERR_DEVICE (-6)
#define SSQA_ERR_NOT_FOUND (-7)

/* --------------------------------------------------------------- options */
#define SSQA_COUPLING_UPPER 0 /* Eq. 6a as printed: J_perp(t) sigma_{i,k+1}(t-d)  */
#define SSQA_COUPLING_BOTH 1  /* adds J_perp(t) sigma_{i,k-1}(t-d) (both ring
                                 neighbours of Fig. 2 / Eq. 4)                  */

#define SSQA_INIT_RANDOM 0     /* sigma(0) from Philox (cycle word 0xFFFFFFFF), Is = 0 */
#define SSQA_INIT_ALL_MINUS 1  /* sigma(0) = -1, Is = 0                              */
#define SSQA_INIT_FROM_STATE 2 /* resume: sigma, sigma_hist and is_state are inputs */

#define SSQA_ALGO_AUTO 0   /* resident tensor path (N <= 512), else the streamed
                              tensor path (N > 256), else delta                     */
#define SSQA_ALGO_PLAIN 1  /* CUDA-core path, one kernel launch per cycle          */
#define SSQA_ALGO_TENSOR 2 /* tcgen05 paths, one persistent launch for all cycles:
                              resident when the instance fits one SM, else
                              streamed; SSQA_ERR_UNSUPPORTED if neither can take it */
#define SSQA_ALGO_DELTA 3  /* CUDA-core path keeping F = J sigma per column and, each
                              cycle, adding only the flipped spins' columns of J (a
                              dense recompute when many flip); AUTO picks it when no
                              tensor path can take the instance                     */
#define SSQA_ALGO_STREAMED 4 /* the streamed tcgen05 path only (N > 256): J streamed
                              from L2 in 256-spin chunks, clusters of up to 16 CTAs
                              per 128 (or 256) spin columns; SSQA_ERR_UNSUPPORTED
                              otherwise                                              */

#define SSQA_FLAG_TRACK_BEST 1u  /* fill e_best / best_cycle                      */
#define SSQA_FLAG_DEVICE_PTRS 2u /* state / result pointers are device pointers  */

/* ------------------------------------------------------------- instances */
/* An Ising instance (Eq. 1): N spins, integer biases h' (int32, length N)
 * and couplings J' (int8, N x N, symmetric, zero diagonal), plus the energy
 * offset e_offset such that (for GI instances) S * H_QUBO(x) = E'(sigma) +
 * e_offset, i.e. the ground energy of an isomorphic pair is -e_offset.
 * Opaque and immutable once built; thread-safe to share between calls. */
typedef struct ssqa_ising ssqa_ising;

/* Erdos-Renyi graph G(n, p), p = p_q32 / 2^32, used to generate GI instances
 * (Sec. 4.2, "Simulation setup").  Generator: SplitMix64 seeded with `seed`;
 * pairs i < j in lexicographic order, one draw each, edge iff the top 32
 * bits of the draw are below p_q32.
 *   adj: caller-owned n*n bytes, row-major; written symmetric, zero diagonal.
 * Errors: SSQA_ERR_INVALID_ARG (n < 1 or n > 65535, adj NULL). */
int ssqa_gen_er_graph(int32_t n, uint32_t p_q32, uint64_t seed, uint8_t *adj);

/* Graph 2 = Graph 1 relabelled by a uniform random permutation pi (Sec. 4.2
 * copies Graph 1 into Graph 2; relabelling hides the planted mapping).
 * Fisher-Yates (i = n-1 .. 1, j uniform in [0, i] from SplitMix64(seed) with
 * rejection of draws >= the largest multiple of i+1 below 2^32).
 *   adj (in, n*n), adj_out (out, n*n): adj_out[pi(u)][pi(v)] = adj[u][v];
 *   perm_out (out, n int32): perm_out[u] = pi(u).
 * Errors: SSQA_ERR_INVALID_ARG. */
int ssqa_permute_graph(int32_t n, const uint8_t *adj, uint64_t seed, uint8_t *adj_out,
                       int32_t *perm_out);

/* Graph-isomorphism Ising instance: the penalty Hamiltonian of Eq. 8 (vertex
 * mapping penalty C1, edge inconsistency penalty C2, sums over ordered vertex
 * pairs), expanded into the upper-triangular QUBO of Eq. 7 and converted to
 * Ising form with sigma = 2x - 1, h_a = -Q_aa/2 - 1/4 sum_{b!=a} Q_ab,
 * J_ab = -Q_ab/4 (Sec. 4.2), everything multiplied by `scale` (S).
 * Spin index a = u*n + i means "vertex u of Graph 2 maps to vertex i of
 * Graph 1"; N = n*n.
 *   adj1, adj2: n*n adjacency bytes (symmetric, zero diagonal) of Graph 1, 2.
 *   C1, C2 > 0; scale > 0 with every scaled value an integer (scale % 4 == 0
 *   always suffices) and every J' in int8 range.
 *   out: receives a library-owned instance; free with ssqa_ising_free.
 * Errors: SSQA_ERR_INVALID_ARG (bad sizes, asymmetric graphs, non-integral or
 * out-of-range scaled values), SSQA_ERR_OOM. */
int ssqa_build_gi_ising(int32_t n, const uint8_t *adj1, const uint8_t *adj2, int32_t C1,
                        int32_t C2, int32_t scale, ssqa_ising **out);

/* Instance from dense integer coefficients (any Ising problem, Eq. 1).
 *   J: N*N int8, row-major, symmetric with zero diagonal (checked);
 *   h: N int32; e_offset: stored as is (0 if unknown).
 *   out: library-owned instance.
 * Errors: SSQA_ERR_INVALID_ARG, SSQA_ERR_OOM. */
int ssqa_ising_from_dense(int32_t N, const int8_t *J, const int32_t *h, int64_t e_offset,
                          ssqa_ising **out);

/* Release an instance and every device copy made of it.  NULL is a no-op.
 * The caller must not release an instance that a pending server request or
 * an in-flight asynchronous call still uses. */
void ssqa_ising_free(ssqa_ising *ising);

/* Read back an instance: N (may be NULL), e_offset (may be NULL), and, if
 * non-NULL, h (N int32) and J (N*N int8) copied into caller buffers.
 * Errors: SSQA_ERR_INVALID_ARG. */
int ssqa_ising_export(const ssqa_ising *ising, int32_t *N, int64_t *e_offset, int32_t *h,
                      int8_t *J);

/* ------------------------------------------------------------- annealing */
/* Parameters of one anneal (Eq. 6 and Table 2), all in scaled integers. */
typedef struct ssqa_params {
    int32_t R;            /* Trotter replicas (Eq. 4-5), 1 .. 128               */
    int32_t cycles;       /* number of updates t -> t+1 to run (SC, Eq. 9), >= 0 */
    int32_t trials;       /* independent anneals, >= 1                          */
    int32_t I0;           /* counter bound I0' (Eq. 6b), 1 .. 16383             */
    int32_t alpha;        /* counter resolution alpha' (Eq. 6b), 1 .. 2*I0      */
    int32_t n_rnd;        /* noise magnitude n_rnd' (Eq. 6a), >= 0              */
    int32_t jperp_min;    /* J_perp schedule of Sec. 4.2 / Table 2: J_perp(t) =  */
    int32_t jperp_max;    /*   jperp_min + floor((t mod tau(beta+1)) / tau)      */
    int32_t beta;         /*   * (jperp_max - jperp_min) / beta; the difference  */
    int32_t tau;          /*   must be divisible by beta; beta, tau >= 1         */
    int32_t delay;        /* d of Eq. 6a, 0 .. 3                                */
    int32_t coupling;     /* SSQA_COUPLING_*                                    */
    int32_t init_mode;    /* SSQA_INIT_*                                        */
    int32_t algo;         /* SSQA_ALGO_*                                        */
    uint32_t flags;       /* SSQA_FLAG_*                                        */
    int32_t start_cycle;  /* t of the first update (0, or the resume point)    */
    uint32_t trial_offset;/* global index of trial 0; trial j uses trial_offset+j
                             in its noise counters, so a run split over several
                             calls or devices equals one run                    */
    uint64_t seed;        /* Philox4x32-10 key (low word, high word)            */
    int32_t i0_max;       /* I0 schedule of SSA (Sec. 4.4): 0 or I0 keeps I0 fixed
                             (SSQA, Table 2); otherwise I0(t) = I0 * i0_mult^l,
                             l = floor((t mod i0_tau L) / i0_tau), L levels up to
                             i0_max = I0 * i0_mult^(L-1)                         */
    int32_t i0_mult;      /*   1/beta of Sec. 4.4 (2 for beta = 0.5), >= 2     */
    int32_t i0_tau;       /*   cycles per I0 level (tau = 10 in Sec. 4.4), >= 1 */
} ssqa_params;

/* Fill `p` with Table 2's constants at S = 12: I0 24, alpha 1, n_rnd 12,
 * J_perp 0 .. 6 in beta = 3 steps, tau = 100, d = 1, upper coupling, random
 * init, AUTO algorithm, no flags, R = 25 (Sec. 4.3), 1 trial, 0 cycles,
 * fixed I0 (i0_max 0, i0_mult 2, i0_tau 10).  SSA (Eq. 2, Sec. 4.4) is the
 * special case R = 1, J_perp = 0 with an I0 schedule. */
void ssqa_params_default(ssqa_params *p);

/* Outputs (and, with SSQA_INIT_FROM_STATE, inputs) of ssqa_anneal.  Layouts
 * are trial-major, then replica, then spin: element (trial, k, i) of a
 * [trials][R][N] array is at (trial*R + k)*N + i.
 *   sigma      [trials][R][N] int8 (+1/-1): out sigma(t0 + cycles);
 *              in sigma(t0) when resuming.                       (required)
 *   sigma_hist [trials][delay][R][N] int8: level l holds sigma(t - 1 - l);
 *              out always, in when resuming; may be NULL if delay == 0 or if
 *              neither resuming nor checkpointing.
 *   is_state   [trials][R][N] int32: counter Is (Eq. 6b), out; in when
 *              resuming.  Required with SSQA_FLAG_DEVICE_PTRS and when
 *              resuming; otherwise may be NULL, and the counters are then
 *              not returned (the anneal itself is unchanged).
 *   e_final    [trials][R] int64: E'(sigma(t0+cycles)) of Eq. 5 per
 *              replica; may be NULL.
 *   e_best     [trials][R] int64 and best_cycle [trials][R] int32: lowest
 *              E' over sigma(t0+1 .. t0+cycles) and the first t reaching it;
 *              written with SSQA_FLAG_TRACK_BEST (both non-NULL then).
 *   e_trace    [cycles][trials][R] int64: E'(sigma(t0 + c + 1)) of every
 *              replica after every cycle c, the energy waveform of Fig. 6
 *              (Sec. 4.3); may be NULL; needs SSQA_FLAG_TRACK_BEST (the same
 *              per-cycle energies).  Not returned by ssqa_poll (serving). */
typedef struct ssqa_result {
    int8_t *sigma;
    int8_t *sigma_hist;
    int32_t *is_state;
    int64_t *e_final;
    int64_t *e_best;
    int32_t *best_cycle;
    int64_t *e_trace;
} ssqa_result;

/* Run SSQA (Eq. 6a-6c, Sec. 3.2) on all N*R spins of every trial in
 * parallel, for `cycles` synchronous updates, with the J_perp schedule of
 * Sec. 4.2 and Philox4x32-10 noise r_{i,k}(t) keyed by (seed; spin block,
 * replica, trial, cycle).  Results are bit-identical whatever the algorithm,
 * batch size or device.
 *   ising: instance; params: see ssqa_params; out: see ssqa_result.
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream).  Host-pointer
 *   calls return after the results are in host memory; device-pointer calls
 *   (SSQA_FLAG_DEVICE_PTRS) only enqueue work on the stream.
 * Errors: SSQA_ERR_INVALID_ARG (parameter out of range, missing buffer),
 * SSQA_ERR_UNSUPPORTED (SSQA_ALGO_TENSOR or SSQA_ALGO_STREAMED forced on an
 * instance whose couplings or size the tensor paths cannot take exactly, or
 * SSQA_ALGO_STREAMED with resumed counters outside -128..127), SSQA_ERR_OOM,
 * SSQA_ERR_DEVICE (no usable GPU, launch or kernel failure). */
int ssqa_anneal(const ssqa_ising *ising, const ssqa_params *params, ssqa_result *out,
                void *cuda_stream);

/* Several independent anneals (Eq. 6 per problem) submitted together: the
 * problems the resident tensor-core kernel takes, of uneven size, cycle
 * count, replica and trial count, seed and instance, run as the column
 * groups of one launch of that kernel (at most 48 problems per launch; one
 * launch per kernel variant: counter format, replica exchange, accumulator,
 * coupling and energy tracking), each CTA with its own problem's
 * parameters.  Batched launches exist for replica delay d = 1 with R dividing
 * 32 (Table 2's d); other problems, and problems for the streamed or
 * CUDA-core paths, run one launch each.  Every problem's result is
 * bit-identical to ssqa_anneal with the same arguments.  Not in the paper,
 * which runs one anneal at a time.
 *   count: problems; isings, params, outs: count entries each, as for
 *   ssqa_anneal; every params[i].flags must include SSQA_FLAG_DEVICE_PTRS
 *   (outs hold device pointers).  The call returns when every problem has
 *   completed on cuda_stream.
 *   launches (may be NULL): receives the number of kernel launches made
 *   (a problem on the streamed or CUDA-core paths may launch more than one
 *   kernel but counts once).
 * Errors: as ssqa_anneal, for the first problem that fails (problems before
 * it may have run). */
int ssqa_anneal_batch(int32_t count, const ssqa_ising *const *isings, const ssqa_params *params,
                      ssqa_result *outs, int32_t *launches, void *cuda_stream);

/* The kernel path ssqa_anneal takes for this instance and these parameters,
 * decided on the host without running anything (no GPU needed).  Not in the
 * paper: it exposes the library's choice between its exact paths for Eq. 6
 * (the resident and streamed tensor-core kernels, whose FP8 field product is
 * exact only while every partial sum of J sigma + h stays an integer within
 * the accumulator's exact range, and the CUDA-core paths).
 *   desc: if non-NULL and len > 0, receives a NUL-terminated one-line
 *   description (truncated to len - 1 bytes): the path and, for the resident
 *   kernel, its accumulator (FP16 when max_i (|h_i| + sum_j |J_ij|) / jm +
 *   max_i |h_i| / jm <= 2048, else FP32 up to 2^14), counter format and
 *   replica exchange.
 * Returns SSQA_ALGO_TENSOR (resident kernel), SSQA_ALGO_STREAMED,
 * SSQA_ALGO_DELTA or SSQA_ALGO_PLAIN; or SSQA_ERR_INVALID_ARG (as for
 * ssqa_anneal) or SSQA_ERR_UNSUPPORTED (a forced tensor path cannot take the
 * problem).  A resumed state whose counters lie outside -128..127 is only seen
 * at run time: AUTO then moves it from the streamed to the delta path. */
int ssqa_plan(const ssqa_ising *ising, const ssqa_params *params, char *desc, size_t len);

/* ssqa_anneal_noalloc -- the plain CUDA-core anneal (the computation of
 * ssqa_anneal with SSQA_ALGO_PLAIN) without any device-memory allocation.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory: plugins whose host framework owns all
 * device memory and forbids cudaMalloc after start-up, real-time loops in
 * which an allocation (which may synchronise the device) would break the
 * timing, and deployments that fix their device footprint at
 * initialisation.
 *   N: spins; J_padded: device, N rows of roundup(N, 16) bytes (row pitch
 *   roundup(N, 16), zero padded), symmetric J' with zero diagonal; h: device,
 *   N int32.  params: as for ssqa_anneal; flags must include
 *   SSQA_FLAG_DEVICE_PTRS (all `out` pointers are device pointers); algo is
 *   ignored.  The call only enqueues work on cuda_stream.
 * Alignment: J_padded 16 bytes; h, is_state and best_cycle 4 bytes; e_final,
 * e_best and e_trace 8 bytes (sigma and sigma_hist are bytes).  A misaligned
 * pointer returns SSQA_ERR_INVALID_ARG before anything is launched.
 * Scratch: one fixed 16 MiB device array inside the library, held on every
 * GPU that loads the library until the process exits.  A problem needing
 * (delay + 2) * trials * R * roundup(N, 16) bytes plus 16 bytes per column
 * (and alignment) beyond that returns SSQA_ERR_INVALID_ARG.  Every call
 * shares the array and re-initialises what it reads, so calls whose work
 * overlaps on the GPU (different streams, or different host threads on the
 * same device) race and must be serialised by the caller.
 * The first call on each device looks up the array's device address (once
 * per device, in the context current at that call, normally the device's
 * primary context); make that first call before any stream capture begins.
 * The cached address is not valid after cudaDeviceReset or in another
 * context: use the entry point only in the context of its first call.
 * Never calls cudaMalloc, cudaFree or any allocating routine.
 * Errors: SSQA_ERR_INVALID_ARG, SSQA_ERR_DEVICE. */
int ssqa_anneal_noalloc(int32_t N, const int8_t *J_padded, const int32_t *h, const ssqa_params *params,
                        ssqa_result *out, void *cuda_stream);

/* Problem energy E'(sigma) = -sum_i h'_i s_i - sum_{i<j} J'_ij s_i s_j
 * (Eq. 1; Eq. 5 per replica) of `count` spin vectors, on the GPU.
 *   sigma: count*N int8 (+1/-1); E_out: count int64.
 *   flags: SSQA_FLAG_DEVICE_PTRS makes both device pointers and the call
 *   asynchronous on cuda_stream.
 * Errors: SSQA_ERR_INVALID_ARG, SSQA_ERR_OOM, SSQA_ERR_DEVICE. */
int ssqa_energy(const ssqa_ising *ising, const int8_t *sigma, int64_t count, int64_t *E_out,
                uint32_t flags, void *cuda_stream);

/* Time to solution, Eq. 10: t ln(1 - p_target) / ln(1 - p_s).  The paper
 * notes it is undefined at p_s = 0 or 1 and tends to 0 as p_s -> 1; the
 * limits are returned: 0 for p_s >= 1, +infinity for p_s <= 0.  NaN for
 * p_target outside (0, 1). */
double ssqa_tts(double t, double p_s, double p_target);

/* Bound of the device-side waits of the tensor-core kernels, in SM clocks.
 * Every wait of a kernel for its tensor cores, its copies or another warp or
 * CTA gives up after this many clocks: the kernel then stops its work, lets
 * its own operations in flight finish (with a fixed bound of 4e9 clocks),
 * frees its tensor memory and returns, and the call reports
 * SSQA_ERR_TIMEOUT; the CUDA context stays usable.  0 restores the default
 * of 8e9 clocks (about 4 s at 2 GHz).  Process-wide; applies to launches made
 * after the call.  Not in the paper: it bounds a failure (a stalled device)
 * instead of hanging.  Errors: SSQA_ERR_INVALID_ARG (clocks < 0). */
int ssqa_set_wait_limit(int64_t clocks);

/* Human-readable description of the last error on this thread ("" if none). */
const char *ssqa_last_error(void);

/* --------------------------------------------------------------- serving */
/* A continuous-batching server: requests are admitted while a slot and
 * enough of the HBM budget are free, run concurrently on the device (one
 * stream per slot, device-resident state for the whole anneal), and are
 * completed in any order.  A request's result is bit-identical to the same
 * ssqa_anneal call made alone.  Not described in the paper (which runs one
 * MATLAB anneal at a time); the per-request computation is Eq. 6. */
typedef struct ssqa_server ssqa_server;

/* hbm_budget: bytes of device memory the server may hold for admitted
 * requests (instance copies, state, results); max_slots: concurrent
 * requests, 1 .. 64; device: CUDA device ordinal.  out: library-owned.
 * Errors: SSQA_ERR_INVALID_ARG, SSQA_ERR_DEVICE, SSQA_ERR_OOM. */
int ssqa_server_create(size_t hbm_budget, int32_t max_slots, int32_t device, ssqa_server **out);

/* Stop accepting work, wait for admitted requests, release everything.
 * NULL is a no-op. */
void ssqa_server_destroy(ssqa_server *server);

/* Queue one anneal.  The instance must stay alive until the request is
 * polled complete; params are copied (SSQA_FLAG_DEVICE_PTRS is rejected:
 * results come back through ssqa_poll into host memory).
 *   ticket: receives an identifier unique within the server.
 * Errors: SSQA_ERR_INVALID_ARG, SSQA_ERR_BUDGET (the request alone needs
 * more than the whole budget). */
int ssqa_submit(ssqa_server *server, const ssqa_ising *ising, const ssqa_params *params,
                uint64_t *ticket);

/* Wait up to timeout_ms (0 = just test, < 0 = forever) for a request.
 * On completion copies the results into `out` (host buffers sized as for
 * ssqa_anneal), forgets the ticket and returns SSQA_OK; returns
 * SSQA_PENDING if it is still queued or running when the time is up.
 *   latency_us (may be NULL): submit-to-completion time in microseconds.
 * Errors: SSQA_ERR_NOT_FOUND (unknown or already collected ticket), or the
 * request's own error code. */
int ssqa_poll(ssqa_server *server, uint64_t ticket, ssqa_result *out, int32_t timeout_ms,
              double *latency_us);

#ifdef __cplusplus
}
#endif
#endif /* SSQA_H */
