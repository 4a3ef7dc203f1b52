// C ABI of the SSQA library: argument checking, instance construction
// (Sec. 4.1-4.2 of the paper), device copies, and dispatch of the anneal to
// the CUDA kernels.  Every step of an anneal runs on the GPU.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "ssqa_internal.h"

namespace ssqa {

static thread_local std::string g_last_error;
static std::atomic<long long> g_wait_clocks{0};

long long wait_limit_clocks() {
    const long long v = g_wait_clocks.load(std::memory_order_relaxed);
    return v > 0 ? v : 8000000000LL;
}

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = pools.find(dev);
        if (it == pools.end()) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if ((e = cudaMemPoolCreate(&pool, &props))) return e;
            int no = 0;
            cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            pools.emplace(dev, pool);
        } else {
            pool = it->second;
        }
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

int check_device(int *device) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SSQA_ERR_DEVICE, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    int major = 0;
    e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e != cudaSuccess || major != 10)
        return fail(SSQA_ERR_DEVICE, "the library is built for sm_103a (compute capability 10.x)");
    if (device) *device = dev;
    return SSQA_OK;
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014): Weyl step then the 64-bit finaliser.
// ---------------------------------------------------------------------------
namespace {
struct SplitMix64 {
    uint64_t s;
    explicit SplitMix64(uint64_t seed) : s(seed) {}
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    // uniform in [0, m): top 32 bits, rejecting the biased tail of 2^32
    uint32_t below(uint32_t m) {
        const uint64_t lim = (uint64_t(1) << 32) - ((uint64_t(1) << 32) % m);
        for (;;) {
            uint64_t x = next() >> 32;
            if (x < lim) return uint32_t(x % m);
        }
    }
};

// FP8 E4M3 (OCP "FN" variant: bias 7, no infinities) encoding of an integer,
// or -1 if it has no exact E4M3 value.
int e4m3_of_int(int64_t v) {
    if (v == 0) return 0;
    int sign = v < 0 ? 0x80 : 0;
    uint64_t a = uint64_t(v < 0 ? -v : v);
    if (a > 448) return -1;
    int e = 63 - __builtin_clzll(a);     // a in [2^e, 2^(e+1))
    uint64_t frac = a - (uint64_t(1) << e);  // mantissa bits: frac / 2^e * 8
    if (e >= 3) {
        if (frac % (uint64_t(1) << (e - 3))) return -1;
        frac >>= (e - 3);
    } else {
        frac <<= (3 - e);
    }
    int biased = e + 7;
    if (biased > 15 || (biased == 15 && frac == 7)) return -1;
    return sign | (biased << 3) | int(frac);
}

int64_t gcd64(int64_t a, int64_t b) {
    a = a < 0 ? -a : a;
    b = b < 0 ? -b : b;
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Build the tcgen05 operand image of an instance (see TcImage).
void prepare_tc(ssqa_ising *I) {
    TcImage &t = I->tc;
    const int N = I->N;
    const size_t NN = size_t(N) * N;
    // J is int8: the common factor, |J| / jm and the FP8 codes are taken once
    // per distinct value (at most 256), then looked up per coupling
    bool present[256] = {};
    for (size_t x = 0; x < NN; ++x) present[uint8_t(I->J[x])] = true;
    int64_t g = 0;
    for (int v = -128; v < 128; ++v)
        if (present[uint8_t(v)]) g = gcd64(g, v);
    for (int32_t v : I->h) g = gcd64(g, v);
    if (g == 0) g = 1;
    if (g > 2048) {
        t.why = "common factor of J and h too large for the FP16 epilogue";
        return;
    }
    t.jm = int32_t(g);
    int64_t mag[256];  // |v / jm| of every int8 value v
    int code[256];     // E4M3 code of v / jm, -1 if none (v = 0 -> 0)
    for (int v = -128; v < 128; ++v) {
        mag[uint8_t(v)] = std::llabs(v / g);
        code[uint8_t(v)] = v % g ? -1 : e4m3_of_int(v / g);
    }
    t.h_unit.resize(N);
    int64_t hmax = 0;
    for (int i = 0; i < N; ++i) {
        t.h_unit[i] = int32_t(I->h[i] / g);
        hmax = std::max<int64_t>(hmax, std::llabs(t.h_unit[i]));
    }
    // h digit columns: weights 1, 16, then 256 repeated
    int nh;
    if (hmax == 0) nh = 0;
    else if (hmax < 16) nh = 1;
    else if (hmax < 256) nh = 2;
    else nh = 2 + int((hmax / 256 + 14) / 15);
    t.nh = nh;
    t.max_h_unit = hmax;
    t.N16 = (N + 15) / 16 * 16;
    t.Kp = (t.N16 + nh + 31) / 32 * 32;
    // accumulator bound: every partial sum of D stays an exact small integer
    for (int i = 0; i < N; ++i) {
        int64_t s = std::llabs(t.h_unit[i]);
        const int8_t *row = I->J.data() + size_t(i) * N;
        for (int j = 0; j < N; ++j) s += mag[uint8_t(row[j])];
        if (s > 16384) {
            t.why = "row sums of |J|/jm + |h|/jm exceed 2^14";
            return;
        }
        t.max_row_sum = std::max(t.max_row_sum, s);
    }
    for (int v = -128; v < 128; ++v)
        if (present[uint8_t(v)] && code[uint8_t(v)] < 0) {
            t.why = "a coupling J/jm has no exact FP8 E4M3 value";
            return;
        }
    t.a_w.assign(nh, 0);
    for (int m = 0; m < nh; ++m) t.a_w[m] = uint8_t(e4m3_of_int(m == 0 ? 1 : (m == 1 ? 16 : 256)));
    auto hdigit = [&](int i, int m) -> uint8_t {
        const int64_t hv = t.h_unit[i];
        const int sgn = hv < 0 ? -1 : 1;
        const int64_t a = std::llabs(hv);
        int64_t d;
        if (m == 0) d = a % 16;
        else if (m == 1) d = (a / 16) % 16;
        else d = std::max<int64_t>(0, std::min<int64_t>(15, a / 256 - int64_t(m - 2) * 15));
        return uint8_t(e4m3_of_int(sgn * d));
    };
    if (N > 256 && nh <= 16) {
        // streamed image: 256-spin chunks x 32-wide K-blocks
        t.KB = t.Kp / 32;
        t.NCH = (t.N16 + 255) / 256;
        t.bs.assign(size_t(t.NCH) * t.KB * 8192, 0);
        auto boff = [&](int i, int k) -> size_t {
            const int ch = i / 256, r = i % 256, kb = k / 32, kk = k % 32;
            return (size_t(ch) * t.KB + kb) * 8192 + size_t(r / 8) * 256 + size_t(kk / 16) * 128 + size_t(r % 8) * 16 +
                   size_t(kk % 16);
        };
        for (int i = 0; i < N; ++i) {
            const int8_t *row = I->J.data() + size_t(i) * N;
            for (int j0 = 0; j0 < N; j0 += 16) {  // 16 consecutive K bytes are contiguous
                uint8_t *dst = t.bs.data() + boff(i, j0);
                const int n = std::min(16, N - j0);
                for (int k = 0; k < n; ++k) dst[k] = uint8_t(code[uint8_t(row[j0 + k])]);
            }
            for (int m = 0; m < nh; ++m) t.bs[boff(i, t.N16 + m)] = hdigit(i, m);
        }
        t.s_ok = true;
    }
    if (N <= 256) {
        t.nchunk = 1;
        t.chunk_rows[0] = t.N16;
    } else if (N <= 512) {
        // the smaller chunk first: its epilogue overlaps the larger chunk's MMAs.
        // About 44 % of the rows balanced best (N = 400: 176 + 224 is 1.9 %
        // faster than 144 + 256); each chunk has at most 256 rows, and the
        // kernel relies on the first one ending at or before spin 256.
        t.nchunk = 2;
        int c0 = (t.N16 * 44 / 100 + 8) / 16 * 16;
        c0 = std::min(256, std::max(c0, t.N16 - 256));
        t.chunk_rows[0] = c0;
        t.chunk_rows[1] = t.N16 - c0;
    } else {
        t.why = "N > 512 needs more tensor memory than one CTA holds";
        return;
    }
    t.Brows = t.chunk_rows[0] + t.chunk_rows[1];
    const int Kp = t.Kp;
    auto off = [Kp](int r, int k) -> size_t {
        return size_t(r / 8) * (size_t(Kp) * 8) + size_t(k / 16) * 128 + size_t(r % 8) * 16 + size_t(k % 16);
    };
    t.b.assign(size_t(t.Brows) * Kp, 0);
    for (int i = 0; i < N; ++i) {
        const int8_t *row = I->J.data() + size_t(i) * N;
        for (int j0 = 0; j0 < N; j0 += 16) {  // 16 consecutive K bytes are contiguous
            uint8_t *dst = t.b.data() + off(i, j0);
            const int n = std::min(16, N - j0);
            for (int k = 0; k < n; ++k) dst[k] = uint8_t(code[uint8_t(row[j0 + k])]);
        }
    }
    for (int i = 0; i < N; ++i)
        for (int m = 0; m < nh; ++m) t.b[off(i, t.N16 + m)] = hdigit(i, m);
    t.ok = true;
}

ssqa_ising *new_ising(int32_t N) {
    ssqa_ising *I = new (std::nothrow) ssqa_ising();
    if (!I) return nullptr;
    try {
        I->N = N;
        I->J.assign(size_t(N) * N, 0);
        I->h.assign(N, 0);
    } catch (...) {
        delete I;
        return nullptr;
    }
    return I;
}
}  // namespace

int device_copy(const ssqa_ising *cI, DeviceCopy **out, cudaStream_t st) {
    ssqa_ising *I = const_cast<ssqa_ising *>(cI);
    int dev = 0;
    int rc = check_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(I->mu);
    auto it = I->dev.find(dev);
    if (it != I->dev.end()) {
        *out = &it->second;
        return SSQA_OK;
    }
    // Stream-ordered allocations from the library pool and copies on the
    // caller's stream, completed before the copy is published (other streams
    // may use it next); ssqa_ising_free returns them with cudaFreeAsync.
    // Neither allocation nor release synchronises the device, so instances can
    // come and go while other anneals run (a server's requests).
    DeviceCopy dc;
    const size_t N = size_t(I->N);
    std::vector<void *> got;
    auto bad = [&](cudaError_t e) {
        for (void *q : got) cudaFreeAsync(q, st);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SSQA_ERR_OOM : SSQA_ERR_DEVICE,
                    std::string("instance upload: ") + cudaGetErrorString(e));
    };
    auto alloc = [&](void **q, size_t bytes) {
        cudaError_t e = dev_alloc(q, bytes ? bytes : 1, st);
        if (!e) got.push_back(*q);
        return e;
    };
    cudaError_t e;
    dc.Np = int32_t((N + 15) / 16 * 16);
    if ((e = alloc(reinterpret_cast<void **>(&dc.J), N * N))) return bad(e);
    if ((e = alloc(reinterpret_cast<void **>(&dc.h), N * 4))) return bad(e);
    if ((e = alloc(reinterpret_cast<void **>(&dc.J_pad), N * dc.Np))) return bad(e);
    if ((e = cudaMemcpyAsync(dc.J, I->J.data(), N * N, cudaMemcpyHostToDevice, st))) return bad(e);
    if ((e = cudaMemsetAsync(dc.J_pad, 0, N * dc.Np, st))) return bad(e);
    if ((e = cudaMemcpy2DAsync(dc.J_pad, dc.Np, I->J.data(), N, N, N, cudaMemcpyHostToDevice, st))) return bad(e);
    if ((e = cudaMemcpyAsync(dc.h, I->h.data(), N * 4, cudaMemcpyHostToDevice, st))) return bad(e);
    std::vector<float> hf;
    if (I->tc.s_ok) {
        if ((e = alloc(reinterpret_cast<void **>(&dc.tcs_b), I->tc.bs.size()))) return bad(e);
        if ((e = cudaMemcpyAsync(dc.tcs_b, I->tc.bs.data(), I->tc.bs.size(), cudaMemcpyHostToDevice, st)))
            return bad(e);
        hf.resize(N);
        for (size_t i = 0; i < N; ++i) hf[i] = float(I->tc.h_unit[i]);
        if ((e = alloc(reinterpret_cast<void **>(&dc.tcs_hf), N * 4))) return bad(e);
        if ((e = cudaMemcpyAsync(dc.tcs_hf, hf.data(), N * 4, cudaMemcpyHostToDevice, st))) return bad(e);
    }
    if (I->tc.ok) {
        if ((e = alloc(reinterpret_cast<void **>(&dc.tc_b), I->tc.b.size()))) return bad(e);
        if ((e = cudaMemcpyAsync(dc.tc_b, I->tc.b.data(), I->tc.b.size(), cudaMemcpyHostToDevice, st))) return bad(e);
        if ((e = alloc(reinterpret_cast<void **>(&dc.tc_h_unit), N * 4))) return bad(e);
        if ((e = cudaMemcpyAsync(dc.tc_h_unit, I->tc.h_unit.data(), N * 4, cudaMemcpyHostToDevice, st)))
            return bad(e);
    }
    if ((e = cudaStreamSynchronize(st))) return bad(e);
    auto res = I->dev.emplace(dev, dc);
    *out = &res.first->second;
    return SSQA_OK;
}

}  // namespace ssqa

using namespace ssqa;

extern "C" {

const char *ssqa_last_error(void) { return g_last_error.c_str(); }

int ssqa_set_wait_limit(int64_t clocks) {
    if (clocks < 0) return fail(SSQA_ERR_INVALID_ARG, "ssqa_set_wait_limit: clocks must be >= 0");
    g_wait_clocks.store(clocks, std::memory_order_relaxed);
    return SSQA_OK;
}

int ssqa_gen_er_graph(int32_t n, uint32_t p_q32, uint64_t seed, uint8_t *adj) {
    if (n < 1 || n > 65535 || !adj) return fail(SSQA_ERR_INVALID_ARG, "ssqa_gen_er_graph: bad n or adj");
    SplitMix64 rng(seed);
    for (int32_t i = 0; i < n; ++i) adj[size_t(i) * n + i] = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j) {
            const uint8_t e = (rng.next() >> 32) < p_q32 ? 1 : 0;
            adj[size_t(i) * n + j] = e;
            adj[size_t(j) * n + i] = e;
        }
    return SSQA_OK;
}

int ssqa_permute_graph(int32_t n, const uint8_t *adj, uint64_t seed, uint8_t *adj_out, int32_t *perm_out) {
    if (n < 1 || n > 65535 || !adj || !adj_out || !perm_out)
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_permute_graph: bad arguments");
    std::vector<int32_t> pi(n);
    std::iota(pi.begin(), pi.end(), 0);
    SplitMix64 rng(seed);
    for (int32_t i = n - 1; i >= 1; --i) std::swap(pi[i], pi[rng.below(uint32_t(i) + 1)]);
    for (int32_t u = 0; u < n; ++u) {
        perm_out[u] = pi[u];
        for (int32_t v = 0; v < n; ++v) adj_out[size_t(pi[u]) * n + pi[v]] = adj[size_t(u) * n + v];
    }
    return SSQA_OK;
}

int ssqa_build_gi_ising(int32_t n, const uint8_t *adj1, const uint8_t *adj2, int32_t C1, int32_t C2,
                        int32_t scale, ssqa_ising **out) {
    if (!out) return fail(SSQA_ERR_INVALID_ARG, "ssqa_build_gi_ising: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 181 || !adj1 || !adj2 || C1 < 1 || C2 < 1 || scale < 1)
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_build_gi_ising: bad n, graph, penalties or scale");
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) {
            const size_t a = size_t(i) * n + j, b = size_t(j) * n + i;
            if (adj1[a] > 1 || adj2[a] > 1 || adj1[a] != adj1[b] || adj2[a] != adj2[b] ||
                (i == j && (adj1[a] || adj2[a])))
                return fail(SSQA_ERR_INVALID_ARG, "ssqa_build_gi_ising: graphs must be 0/1, symmetric, loop-free");
        }
    const int32_t N = n * n;
    // Q of Eq. 7 from Eq. 8, per unordered spin pair {a = (u,i), b = (v,j)}:
    //   same u, i != j  : 2 C1           (square of the row one-hot term)
    //   same i, u != v  : 2 C1           (square of the column one-hot term)
    //   u != v, i != j  : 2 C2 if edge(i,j in G1) != edge(u,v in G2)
    //                     (each mismatch appears as two ordered pairs)
    //   diagonal Q_aa   : -2 C1,  constant 2 n C1.
    // Ising (Sec. 4.2): J_ab = -Q_ab / 4, h_a = -Q_aa/2 - sum_b Q_ab / 4.
    // Everything is carried times 4 and divided by 4 once, after scaling.
    std::unique_ptr<ssqa_ising> I(new_ising(N));
    if (!I) return fail(SSQA_ERR_OOM, "ssqa_build_gi_ising: out of host memory");
    const int64_t S = scale;
    int64_t off4 = 4 * int64_t(2) * n * C1;  // 4 * constant
    for (int32_t u = 0; u < n; ++u)
        for (int32_t i = 0; i < n; ++i) {
            const int32_t a = u * n + i;
            const int64_t qaa = -2 * int64_t(C1);
            int64_t h4 = -2 * qaa;  // 4 * (-Q_aa / 2)
            off4 += 2 * qaa;        // 4 * Q_aa / 2
            for (int32_t v = 0; v < n; ++v)
                for (int32_t j = 0; j < n; ++j) {
                    const int32_t b = v * n + j;
                    if (b == a) continue;
                    int64_t q = 0;
                    if (u == v) q = 2 * int64_t(C1);
                    else if (i == j) q = 2 * int64_t(C1);
                    else if (adj1[size_t(i) * n + j] != adj2[size_t(u) * n + v]) q = 2 * int64_t(C2);
                    if (!q) continue;
                    h4 -= q;
                    if (b > a) off4 += q;
                    const int64_t j4 = -S * q;
                    if (j4 % 4 || j4 / 4 < -127 || j4 / 4 > 127)
                        return fail(SSQA_ERR_INVALID_ARG, "ssqa_build_gi_ising: scaled J not an int8 integer");
                    I->J[size_t(a) * N + b] = int8_t(j4 / 4);
                }
            const int64_t hs = S * h4;
            if (hs % 4 || hs / 4 < INT32_MIN || hs / 4 > INT32_MAX)
                return fail(SSQA_ERR_INVALID_ARG, "ssqa_build_gi_ising: scaled h not an int32 integer");
            I->h[a] = int32_t(hs / 4);
        }
    if ((S * off4) % 4) return fail(SSQA_ERR_INVALID_ARG, "ssqa_build_gi_ising: scaled offset not an integer");
    I->e_offset = S * off4 / 4;
    prepare_tc(I.get());
    *out = I.release();
    return SSQA_OK;
}

int ssqa_ising_from_dense(int32_t N, const int8_t *J, const int32_t *h, int64_t e_offset, ssqa_ising **out) {
    if (!out) return fail(SSQA_ERR_INVALID_ARG, "ssqa_ising_from_dense: out is NULL");
    *out = nullptr;
    if (N < 1 || N > 65536 || !J || !h) return fail(SSQA_ERR_INVALID_ARG, "ssqa_ising_from_dense: bad N, J or h");
    for (int32_t i = 0; i < N; ++i)
        if (J[size_t(i) * N + i]) return fail(SSQA_ERR_INVALID_ARG, "ssqa_ising_from_dense: J diagonal must be 0");
    // symmetry, compared in 32 x 32 tiles (both tiles stay in cache)
    for (int32_t i0 = 0; i0 < N; i0 += 32)
        for (int32_t j0 = i0; j0 < N; j0 += 32) {
            bool sym = true;
            for (int32_t i = i0; i < std::min(i0 + 32, N); ++i)
                for (int32_t j = j0; j < std::min(j0 + 32, N); ++j)
                    sym &= J[size_t(i) * N + j] == J[size_t(j) * N + i];
            if (!sym) return fail(SSQA_ERR_INVALID_ARG, "ssqa_ising_from_dense: J must be symmetric");
        }
    std::unique_ptr<ssqa_ising> I(new_ising(N));
    if (!I) return fail(SSQA_ERR_OOM, "ssqa_ising_from_dense: out of host memory");
    std::memcpy(I->J.data(), J, size_t(N) * N);
    std::memcpy(I->h.data(), h, size_t(N) * 4);
    I->e_offset = e_offset;
    prepare_tc(I.get());
    *out = I.release();
    return SSQA_OK;
}

void ssqa_ising_free(ssqa_ising *I) {
    if (!I) return;
    int cur = 0;
    cudaGetDevice(&cur);
    // the memory returns to the library pool in the legacy stream's order:
    // no device-wide synchronisation (the caller guarantees no work still
    // uses the instance)
    for (auto &kv : I->dev) {
        cudaSetDevice(kv.first);
        void *ps[] = {kv.second.J, kv.second.J_pad, kv.second.h, kv.second.tc_b, kv.second.tc_h_unit,
                      kv.second.tcs_b, kv.second.tcs_hf};
        for (void *q : ps)
            if (q) cudaFreeAsync(q, nullptr);
    }
    cudaSetDevice(cur);
    cudaGetLastError();
    delete I;
}

int ssqa_ising_export(const ssqa_ising *I, int32_t *N, int64_t *e_offset, int32_t *h, int8_t *J) {
    if (!I) return fail(SSQA_ERR_INVALID_ARG, "ssqa_ising_export: NULL instance");
    if (N) *N = I->N;
    if (e_offset) *e_offset = I->e_offset;
    if (h) std::memcpy(h, I->h.data(), size_t(I->N) * 4);
    if (J) std::memcpy(J, I->J.data(), size_t(I->N) * I->N);
    return SSQA_OK;
}

void ssqa_params_default(ssqa_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->R = 25;
    p->cycles = 0;
    p->trials = 1;
    p->I0 = 24;
    p->alpha = 1;
    p->n_rnd = 12;
    p->jperp_min = 0;
    p->jperp_max = 6;
    p->beta = 3;
    p->tau = 100;
    p->delay = 1;
    p->coupling = SSQA_COUPLING_UPPER;
    p->init_mode = SSQA_INIT_RANDOM;
    p->algo = SSQA_ALGO_AUTO;
    p->i0_max = 0;
    p->i0_mult = 2;
    p->i0_tau = 10;
}

double ssqa_tts(double t, double p_s, double p_target) {
    if (!(p_target > 0.0 && p_target < 1.0)) return std::numeric_limits<double>::quiet_NaN();
    if (p_s >= 1.0) return 0.0;
    if (p_s <= 0.0) return std::numeric_limits<double>::infinity();
    return t * std::log1p(-p_target) / std::log1p(-p_s);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// anneal / energy dispatch
// ---------------------------------------------------------------------------
namespace {

int validate(const ssqa_ising *I, const ssqa_params *p, const ssqa_result *r) {
    if (!I || !p || !r) return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal: NULL argument");
    if (p->R < 1 || p->R > 128) return fail(SSQA_ERR_INVALID_ARG, "R must be in 1..128");
    if (p->trials < 1 || p->cycles < 0) return fail(SSQA_ERR_INVALID_ARG, "trials >= 1 and cycles >= 0 required");
    if (int64_t(p->trials) * p->R > (int64_t(1) << 30) ||
        int64_t(p->trials) * p->R * I->N > (int64_t(1) << 40))
        return fail(SSQA_ERR_INVALID_ARG, "trials * R * N too large");
    if (p->I0 < 1 || p->I0 > 16383) return fail(SSQA_ERR_INVALID_ARG, "I0 must be in 1..16383");
    if (p->alpha < 1 || p->alpha > 2 * p->I0) return fail(SSQA_ERR_INVALID_ARG, "alpha must be in 1..2*I0");
    if (p->n_rnd < 0 || p->n_rnd > (1 << 20)) return fail(SSQA_ERR_INVALID_ARG, "n_rnd out of range");
    if (p->beta < 1 || p->tau < 1) return fail(SSQA_ERR_INVALID_ARG, "beta and tau must be >= 1");
    if (std::abs(int64_t(p->jperp_min)) > (1 << 20) || std::abs(int64_t(p->jperp_max)) > (1 << 20))
        return fail(SSQA_ERR_INVALID_ARG, "jperp out of range");
    if ((int64_t(p->jperp_max) - p->jperp_min) % p->beta)
        return fail(SSQA_ERR_INVALID_ARG, "(jperp_max - jperp_min) must be divisible by beta");
    if (p->delay < 0 || p->delay > 3) return fail(SSQA_ERR_INVALID_ARG, "delay must be in 0..3");
    if (p->coupling != SSQA_COUPLING_UPPER && p->coupling != SSQA_COUPLING_BOTH)
        return fail(SSQA_ERR_INVALID_ARG, "unknown coupling mode");
    if (p->init_mode < 0 || p->init_mode > 2) return fail(SSQA_ERR_INVALID_ARG, "unknown init mode");
    if (p->algo < 0 || p->algo > 4) return fail(SSQA_ERR_INVALID_ARG, "unknown algo");
    if (p->start_cycle < 0 || int64_t(p->start_cycle) + p->cycles > 0xFFFFFFFEll)
        return fail(SSQA_ERR_INVALID_ARG, "cycle range must stay below 2^32 - 1");
    if (int64_t(p->trial_offset) + p->trials > 0xFFFFFFFFll)
        return fail(SSQA_ERR_INVALID_ARG, "trial_offset + trials must fit 32 bits");
    if (!r->sigma) return fail(SSQA_ERR_INVALID_ARG, "the sigma buffer is required");
    if (!r->is_state && ((p->flags & SSQA_FLAG_DEVICE_PTRS) || p->init_mode == SSQA_INIT_FROM_STATE))
        return fail(SSQA_ERR_INVALID_ARG, "is_state is required with device pointers and when resuming");
    if (p->init_mode == SSQA_INIT_FROM_STATE && p->delay > 0 && !r->sigma_hist)
        return fail(SSQA_ERR_INVALID_ARG, "resuming with delay > 0 needs sigma_hist");
    if ((p->flags & SSQA_FLAG_TRACK_BEST) && (!r->e_best || !r->best_cycle))
        return fail(SSQA_ERR_INVALID_ARG, "TRACK_BEST needs e_best and best_cycle");
    if (r->e_trace && !(p->flags & SSQA_FLAG_TRACK_BEST))
        return fail(SSQA_ERR_INVALID_ARG, "e_trace needs SSQA_FLAG_TRACK_BEST");
    if (p->flags & ~(SSQA_FLAG_TRACK_BEST | SSQA_FLAG_DEVICE_PTRS))
        return fail(SSQA_ERR_INVALID_ARG, "unknown flag bits");
    if (p->i0_max > p->I0) {
        if (p->i0_mult < 2 || p->i0_tau < 1 || p->i0_max > 16383)
            return fail(SSQA_ERR_INVALID_ARG, "I0 schedule: i0_mult >= 2, i0_tau >= 1, i0_max <= 16383");
        int64_t v = p->I0;
        while (v < p->i0_max) v *= p->i0_mult;
        if (v != p->i0_max) return fail(SSQA_ERR_INVALID_ARG, "I0 schedule: i0_max must be I0 * i0_mult^m");
        if (p->alpha > 2 * p->I0) return fail(SSQA_ERR_INVALID_ARG, "alpha must be in 1..2*I0");
    }
    return SSQA_OK;
}

// Launch arguments of an anneal (instance pointers and buffers left empty).
AnnealArgs make_args(const ssqa_ising *I, const ssqa_params *p) {
    AnnealArgs a{};
    a.N = I->N;
    a.R = p->R;
    a.trials = p->trials;
    a.cycles = p->cycles;
    a.I0 = p->I0;
    a.alpha = p->alpha;
    a.n_rnd = p->n_rnd;
    a.jperp_min = p->jperp_min;
    a.jperp_step = (p->jperp_max - p->jperp_min) / p->beta;
    a.beta = p->beta;
    a.tau = p->tau;
    a.delay = p->delay;
    a.both = p->coupling == SSQA_COUPLING_BOTH;
    a.init_mode = p->init_mode;
    a.start_cycle = p->start_cycle;
    a.trial_offset = p->trial_offset;
    a.seed = p->seed;
    a.i0_max = p->i0_max;
    a.i0_mult = p->i0_mult;
    a.i0_tau = p->i0_tau;
    a.track_best = p->flags & SSQA_FLAG_TRACK_BEST;
    a.Np = (I->N + 15) / 16 * 16;
    return a;
}

// The kernel path an anneal takes (host decision; no device work).  The
// streamed path can still hand a resumed state whose counters do not fit a
// byte back to the CUDA-core paths at run time (AUTO only).
int choose_path(const ssqa_ising *I, const ssqa_params *p, const AnnealArgs &a, int *algo, std::string *desc) {
    std::string why, why_s;
    if (p->algo == SSQA_ALGO_PLAIN) {
        *algo = SSQA_ALGO_PLAIN;
        *desc = "plain CUDA-core path (dp4a), one launch per cycle";
        return SSQA_OK;
    }
    if (p->algo == SSQA_ALGO_DELTA) {
        *algo = SSQA_ALGO_DELTA;
        *desc = "delta-field CUDA-core path";
        return SSQA_OK;
    }
    bool use_tc = false, use_tcs = false;
    if (p->algo == SSQA_ALGO_STREAMED) {
        use_tcs = tcs_supported(I->tc, a, &why_s);
        if (!use_tcs) return fail(SSQA_ERR_UNSUPPORTED, "streamed tensor path: " + why_s);
    } else {
        use_tc = tc_supported(I->tc, a, &why);
        if (!use_tc) use_tcs = tcs_supported(I->tc, a, &why_s);
        if (p->algo == SSQA_ALGO_TENSOR && !use_tc && !use_tcs)
            return fail(SSQA_ERR_UNSUPPORTED, "tensor path: " + why + "; streamed tensor path: " + why_s);
    }
    if (use_tc) {
        const TcVariant v = tc_variant(I->tc, a);
        *algo = SSQA_ALGO_TENSOR;
        *desc = std::string("resident tcgen05 kernel, ") + (v.f16 ? "FP16" : "FP32") + " accumulator, " +
                (v.bytes ? "byte" : "half2") + " counters, " + (v.shfl ? "shuffle" : "shared-memory") +
                " replica exchange";
    } else if (use_tcs) {
        *algo = SSQA_ALGO_STREAMED;
        int dev = 0, nsm = 148;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            nsm = 148;
        }
        const int64_t groups = (int64_t(a.trials) + 128 / a.R - 1) / (128 / a.R);
        const bool dual = I->tc.KB >= 160;
        const int cs = tcs_cluster_size(I->tc, a, nsm);
        *desc = std::string("streamed tcgen05 kernel, FP32 accumulator, ") +
                (dual ? "two column groups per CTA" : "one column group per CTA") + " (groups " +
                std::to_string(groups) + ", KB " + std::to_string(I->tc.KB) + ", NCH " + std::to_string(I->tc.NCH) +
                ", CS " + std::to_string(cs) + ", dual " + (dual ? "1" : "0") + ", CTAs " +
                std::to_string((dual ? (groups + 1) / 2 : groups) * cs) + ")";
    } else {
        *algo = SSQA_ALGO_DELTA;
        *desc = "delta-field CUDA-core path (no tensor path takes this problem: " + why +
                (why_s.empty() || why_s == why ? std::string() : "; " + why_s) + ")";
    }
    return SSQA_OK;
}

struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, s);
    }
};

int cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? SSQA_ERR_OOM : SSQA_ERR_DEVICE,
                std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

namespace {
// A named range on the calling thread's NVTX stack for the span of one entry
// point (shown by profilers that record NVTX; a no-op without one).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace

extern "C" int ssqa_anneal(const ssqa_ising *I, const ssqa_params *p, ssqa_result *r, void *stream) {
    const Range range("ssqa_anneal");
    int rc = validate(I, p, r);
    if (rc) return rc;
    DeviceCopy *dc = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = device_copy(I, &dc, st))) return rc;
    const bool devptr = p->flags & SSQA_FLAG_DEVICE_PTRS;
    const size_t cols = size_t(p->trials) * p->R;
    const size_t nsp = cols * I->N;
    const int d = p->delay;

    AnnealArgs a = make_args(I, p);
    a.J = dc->J;
    a.J_pad = dc->J_pad;
    a.Np = dc->Np;
    a.h = dc->h;

    // state / result buffers on the device
    DevBuf b_sig, b_hist, b_is, b_ef, b_eb, b_bc, b_tr;
    auto alloc = [&](DevBuf &b, size_t bytes) -> cudaError_t {
        b.s = st;
        return dev_alloc(&b.p, bytes ? bytes : 1, st);
    };
    cudaError_t e;
    if (devptr) {
        a.sigma = r->sigma;
        a.hist = d ? r->sigma_hist : nullptr;
        a.Is = r->is_state;
        a.e_final = r->e_final;
        a.e_best = a.track_best ? r->e_best : nullptr;
        a.best_cycle = a.track_best ? r->best_cycle : nullptr;
        a.e_trace = r->e_trace;
    } else {
        if ((e = alloc(b_sig, nsp))) return cuda_fail(e, "ssqa_anneal: state allocation");
        if ((e = alloc(b_is, nsp * 4))) return cuda_fail(e, "ssqa_anneal: state allocation");
        a.sigma = static_cast<int8_t *>(b_sig.p);
        a.Is = static_cast<int32_t *>(b_is.p);
        if (d && (r->sigma_hist || p->init_mode == SSQA_INIT_FROM_STATE)) {
            if ((e = alloc(b_hist, nsp * d))) return cuda_fail(e, "ssqa_anneal: state allocation");
            a.hist = static_cast<int8_t *>(b_hist.p);
        }
        if (r->e_final) {
            if ((e = alloc(b_ef, cols * 8))) return cuda_fail(e, "ssqa_anneal: result allocation");
            a.e_final = static_cast<int64_t *>(b_ef.p);
        }
        if (a.track_best) {
            if ((e = alloc(b_eb, cols * 8))) return cuda_fail(e, "ssqa_anneal: result allocation");
            if ((e = alloc(b_bc, cols * 4))) return cuda_fail(e, "ssqa_anneal: result allocation");
            a.e_best = static_cast<int64_t *>(b_eb.p);
            a.best_cycle = static_cast<int32_t *>(b_bc.p);
        }
        if (r->e_trace) {
            if ((e = alloc(b_tr, size_t(p->cycles) * cols * 8))) return cuda_fail(e, "ssqa_anneal: trace allocation");
            a.e_trace = static_cast<int64_t *>(b_tr.p);
        }
        if (p->init_mode == SSQA_INIT_FROM_STATE) {
            if ((e = cudaMemcpyAsync(a.sigma, r->sigma, nsp, cudaMemcpyHostToDevice, st)) ||
                (e = cudaMemcpyAsync(a.Is, r->is_state, nsp * 4, cudaMemcpyHostToDevice, st)))
                return cuda_fail(e, "ssqa_anneal: state upload");
            if (d && (e = cudaMemcpyAsync(a.hist, r->sigma_hist, nsp * d, cudaMemcpyHostToDevice, st)))
                return cuda_fail(e, "ssqa_anneal: state upload");
        }
    }

    int algo = SSQA_ALGO_AUTO;
    std::string desc;
    if ((rc = choose_path(I, p, a, &algo, &desc))) return rc;
    const bool use_tc = algo == SSQA_ALGO_TENSOR, use_tcs = algo == SSQA_ALGO_STREAMED;
    bool done = false;
    if (use_tc) {
        rc = tc_anneal(I->tc, *dc, a, st);
        done = true;
    } else if (use_tcs) {
        DevBuf scratch;
        if ((e = alloc(scratch, tcs_scratch_bytes(I->tc, a)))) return cuda_fail(e, "ssqa_anneal: scratch allocation");
        rc = tcs_anneal(I->tc, *dc, a, scratch.p, st);
        // a resumed state the byte counters cannot hold falls back to the CUDA-core paths
        done = !(rc == SSQA_ERR_UNSUPPORTED && p->algo == SSQA_ALGO_AUTO);
    }
    if (!done && algo == SSQA_ALGO_PLAIN) {
        DevBuf scratch;
        if ((e = alloc(scratch, plain_scratch_bytes(a)))) return cuda_fail(e, "ssqa_anneal: scratch allocation");
        rc = plain_anneal(a, scratch.p, st);
    } else if (!done) {
        DevBuf scratch;
        if ((e = alloc(scratch, delta_scratch_bytes(a)))) return cuda_fail(e, "ssqa_anneal: scratch allocation");
        rc = delta_anneal(a, scratch.p, st);
    }
    if (rc) return rc;
    if (!devptr) {
        if ((e = cudaMemcpyAsync(r->sigma, a.sigma, nsp, cudaMemcpyDeviceToHost, st)) ||
            (r->is_state && (e = cudaMemcpyAsync(r->is_state, a.Is, nsp * 4, cudaMemcpyDeviceToHost, st))))
            return cuda_fail(e, "ssqa_anneal: result download");
        if (r->sigma_hist && a.hist &&
            (e = cudaMemcpyAsync(r->sigma_hist, a.hist, nsp * d, cudaMemcpyDeviceToHost, st)))
            return cuda_fail(e, "ssqa_anneal: result download");
        if (r->e_final && (e = cudaMemcpyAsync(r->e_final, a.e_final, cols * 8, cudaMemcpyDeviceToHost, st)))
            return cuda_fail(e, "ssqa_anneal: result download");
        if (a.track_best &&
            ((e = cudaMemcpyAsync(r->e_best, a.e_best, cols * 8, cudaMemcpyDeviceToHost, st)) ||
             (e = cudaMemcpyAsync(r->best_cycle, a.best_cycle, cols * 4, cudaMemcpyDeviceToHost, st))))
            return cuda_fail(e, "ssqa_anneal: result download");
        if (r->e_trace && p->cycles > 0 &&
            (e = cudaMemcpyAsync(r->e_trace, a.e_trace, size_t(p->cycles) * cols * 8, cudaMemcpyDeviceToHost, st)))
            return cuda_fail(e, "ssqa_anneal: result download");
        if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "ssqa_anneal");
    }
    if ((e = cudaGetLastError())) return cuda_fail(e, "ssqa_anneal");
    return SSQA_OK;
}

namespace ssqa {
int batch_key(const ssqa_ising *I, const ssqa_params *p) {
    if (!I || !p || p->R < 1 || p->R > 128 || p->trials < 1 || p->beta < 1) return -1;
    const AnnealArgs a = make_args(I, p);
    int algo = SSQA_ALGO_AUTO;
    std::string desc;
    const std::string saved = g_last_error;
    const int rc = choose_path(I, p, a, &algo, &desc);
    g_last_error = saved;
    if (rc || algo != SSQA_ALGO_TENSOR) return -1;
    return tc_batch_key(I->tc, a);
}
}  // namespace ssqa

extern "C" int ssqa_anneal_batch(int32_t count, const ssqa_ising *const *isings, const ssqa_params *params,
                                 ssqa_result *outs, int32_t *launches, void *stream) {
    const Range range("ssqa_anneal_batch");
    if (launches) *launches = 0;
    if (count < 0 || (count > 0 && (!isings || !params || !outs)))
        return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_batch: bad count or NULL array");
    std::vector<TcBatchItem> batch;
    std::vector<int> single;
    batch.reserve(size_t(count));
    for (int32_t i = 0; i < count; ++i) {
        const ssqa_ising *I = isings[i];
        const ssqa_params *p = &params[i];
        int rc = validate(I, p, &outs[i]);
        if (rc) return rc;
        if (!(p->flags & SSQA_FLAG_DEVICE_PTRS))
            return fail(SSQA_ERR_INVALID_ARG, "ssqa_anneal_batch: every item needs SSQA_FLAG_DEVICE_PTRS");
        DeviceCopy *dc = nullptr;
        if ((rc = device_copy(I, &dc, static_cast<cudaStream_t>(stream)))) return rc;
        AnnealArgs a = make_args(I, p);
        a.J = dc->J;
        a.J_pad = dc->J_pad;
        a.Np = dc->Np;
        a.h = dc->h;
        a.sigma = outs[i].sigma;
        a.hist = p->delay ? outs[i].sigma_hist : nullptr;
        a.Is = outs[i].is_state;
        a.e_final = outs[i].e_final;
        a.e_best = a.track_best ? outs[i].e_best : nullptr;
        a.best_cycle = a.track_best ? outs[i].best_cycle : nullptr;
        a.e_trace = outs[i].e_trace;
        int algo = SSQA_ALGO_AUTO;
        std::string desc;
        if ((rc = choose_path(I, p, a, &algo, &desc))) return rc;
        if (algo == SSQA_ALGO_TENSOR)
            batch.push_back(TcBatchItem{&I->tc, dc, a});
        else
            single.push_back(i);
    }
    int n = 0;
    if (!batch.empty()) {
        if (int rc = tc_anneal_batch(batch.data(), int(batch.size()), &n, stream)) return rc;
    }
    for (int i : single) {
        if (int rc = ssqa_anneal(isings[i], &params[i], &outs[i], stream)) return rc;
        ++n;
    }
    if (launches) *launches = n;
    return SSQA_OK;
}

extern "C" int ssqa_plan(const ssqa_ising *I, const ssqa_params *p, char *desc, size_t len) {
    if (!I || !p) return fail(SSQA_ERR_INVALID_ARG, "ssqa_plan: NULL argument");
    ssqa_result dummy{};
    int8_t one = 0;
    int32_t is = 0;
    int64_t e = 0;
    int32_t bc = 0;
    dummy.sigma = &one;
    dummy.is_state = &is;
    dummy.sigma_hist = &one;
    dummy.e_best = &e;
    dummy.best_cycle = &bc;
    int rc = validate(I, p, &dummy);
    if (rc) return rc;
    const AnnealArgs a = make_args(I, p);
    int algo = SSQA_ALGO_AUTO;
    std::string d;
    if ((rc = choose_path(I, p, a, &algo, &d))) return rc;
    if (desc && len) {
        const size_t n = std::min(len - 1, d.size());
        std::memcpy(desc, d.data(), n);
        desc[n] = 0;
    }
    return algo;
}

extern "C" int ssqa_energy(const ssqa_ising *I, const int8_t *sigma, int64_t count, int64_t *E_out, uint32_t flags,
                           void *stream) {
    const Range range("ssqa_energy");
    if (!I || !sigma || !E_out || count < 0) return fail(SSQA_ERR_INVALID_ARG, "ssqa_energy: bad arguments");
    if (flags & ~uint32_t(SSQA_FLAG_DEVICE_PTRS)) return fail(SSQA_ERR_INVALID_ARG, "ssqa_energy: unknown flags");
    if (count == 0) return SSQA_OK;
    DeviceCopy *dc = nullptr;
    int rc = device_copy(I, &dc, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (flags & SSQA_FLAG_DEVICE_PTRS)
        return energy_launch(dc->J_pad, dc->Np, dc->h, I->N, sigma, I->N, count, E_out, st);
    DevBuf bs, be;
    bs.s = be.s = st;
    const size_t nb = size_t(count) * I->N;
    if ((e = dev_alloc(&bs.p, nb, st)) || (e = dev_alloc(&be.p, size_t(count) * 8, st)))
        return cuda_fail(e, "ssqa_energy: allocation");
    if ((e = cudaMemcpyAsync(bs.p, sigma, nb, cudaMemcpyHostToDevice, st))) return cuda_fail(e, "ssqa_energy: upload");
    rc = energy_launch(dc->J_pad, dc->Np, dc->h, I->N, static_cast<int8_t *>(bs.p), I->N, count,
                       static_cast<int64_t *>(be.p), st);
    if (rc) return rc;
    if ((e = cudaMemcpyAsync(E_out, be.p, size_t(count) * 8, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "ssqa_energy: download");
    return SSQA_OK;
}
