/*
 * ssqa_oracle.c -- plain, slow, single-threaded reference of Stochastic
 * Simulated Quantum Annealing (SSQA, Onizawa et al., arXiv 2302.12454).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include,
 * link or call this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Every function follows one passage of the paper, cited beside it:
 *   - Ising Hamiltonian ............................ Sec. 2.1, Eq. 1
 *   - SSA spin update with an I0 schedule ........... Sec. 2.2, Eq. 2a-2c
 *                                                     (schedule: Sec. 4.4)
 *   - QMC replicas with ring coupling .............. Sec. 3.1, Eq. 4-5
 *   - SSQA spin update ............................. Sec. 3.2, Eq. 6a-6c
 *   - J_perp schedule .............................. Sec. 4.2, Table 2
 *   - QUBO, GI penalty Hamiltonian ................. Sec. 4.1, Eq. 7-8
 *   - QUBO -> Ising conversion ..................... Sec. 4.2 (first paragraph)
 *   - Equivalent cycles, iterations ................ Sec. 4.2, Eq. 9, Table 2
 *   - Time to solution ............................. Sec. 4.3, Eq. 10
 *
 * The paper leaves the random generator, the graph generator and the
 * integer scaling open; the readings taken here are:
 *   - all real-valued quantities are carried as integers scaled by S
 *     (h' = S h, J' = S J, I0' = S I0, n_rnd' = S n_rnd, J_perp' = S J_perp,
 *     alpha' = 1 LSB); with S = 12 every value of Table 2 is an integer;
 *   - the noise r_{i,k}(t) in {-1,+1} is drawn per (spin, replica, trial,
 *     cycle) from Philox4x32-10 (Salmon et al., SC'11).  Spins are grouped
 *     in 32-spin words w = i / 32; word w takes output word (w / 4) % 4 of
 *     the Philox call with counter (4 (w / 16) + w % 4, k, trial, t) and key
 *     (seed low word, seed high word), so one call serves words
 *     {16 j + q, 16 j + q + 4, 16 j + q + 8, 16 j + q + 12}; inside its word,
 *     spin i takes bit 15 - e/2 for even e = i % 32 and bit 31 - (e-1)/2 for
 *     odd e; a set bit means r = -1;
 *   - sigma(0) uses the same bit with t = 0xFFFFFFFF (set bit: sigma = -1),
 *     Is(0) = 0, and sigma(t - d) = sigma(0) for t < d;
 *   - random graphs come from SplitMix64 (Steele, Lea, Flood, OOPSLA'14).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* SplitMix64: state += golden gamma, then the published 64-bit mix.          */
/* ------------------------------------------------------------------------- */
uint64_t or_splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ull;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform integer in [0, m) from the top 32 bits of SplitMix64 outputs,
 * rejecting draws at or above the largest multiple of m below 2^32. */
static uint32_t or_bounded(uint64_t *state, uint32_t m)
{
    uint64_t limit = (0x100000000ull / m) * m;
    for (;;) {
        uint64_t x = or_splitmix64_next(state) >> 32;
        if (x < limit)
            return (uint32_t)(x % m);
    }
}

/* Erdos-Renyi G(n, p) with p = p_q32 / 2^32, the GI instance of Sec. 4.2:
 * pairs i < j in lexicographic order, one draw each, edge iff the draw's top
 * 32 bits are below p_q32.  adj is n*n, symmetric, zero diagonal. */
int or_gen_er_graph(int n, uint32_t p_q32, uint64_t seed, uint8_t *adj)
{
    uint64_t st = seed;
    int i, j;
    if (n < 1 || !adj)
        return -1;
    memset(adj, 0, (size_t)n * n);
    for (i = 0; i < n; ++i)
        for (j = i + 1; j < n; ++j) {
            uint8_t e = (uint8_t)((or_splitmix64_next(&st) >> 32) < p_q32);
            adj[i * n + j] = e;
            adj[j * n + i] = e;
        }
    return 0;
}

/* Graph 2 = Graph 1 relabelled by a random permutation pi (Fisher-Yates,
 * i = n-1 .. 1, swap with a uniform j in [0, i]):
 * adj_out[pi(u)][pi(v)] = adj[u][v], perm_out[u] = pi(u). */
int or_permute_graph(int n, const uint8_t *adj, uint64_t seed, uint8_t *adj_out,
                     int32_t *perm_out)
{
    uint64_t st = seed;
    int i, u, v;
    if (n < 1 || !adj || !adj_out || !perm_out)
        return -1;
    for (i = 0; i < n; ++i)
        perm_out[i] = i;
    for (i = n - 1; i >= 1; --i) {
        int j = (int)or_bounded(&st, (uint32_t)(i + 1));
        int32_t tmp = perm_out[i];
        perm_out[i] = perm_out[j];
        perm_out[j] = tmp;
    }
    for (u = 0; u < n; ++u)
        for (v = 0; v < n; ++v)
            adj_out[perm_out[u] * n + perm_out[v]] = adj[u * n + v];
    return 0;
}

/* ------------------------------------------------------------------------- */
/* GI QUBO, Eq. 8.  Binary x_{u,i} maps vertex u of Graph 2 to vertex i of    */
/* Graph 1; spin index a = u*n + i, N = n^2.  Q is N*N, only a <= b used.     */
/* ------------------------------------------------------------------------- */
static void or_q_add(int64_t *Q, int N, int a, int b, int64_t v)
{
    if (a <= b)
        Q[(size_t)a * N + b] += v;
    else
        Q[(size_t)b * N + a] += v;
}

/* Eq. 8 evaluated term by term for one assignment x (n*n bytes, 0/1). */
int64_t or_gi_hamiltonian(int n, const uint8_t *adj1, const uint8_t *adj2,
                          int64_t C1, int64_t C2, const uint8_t *x)
{
    int64_t H = 0;
    int u, v, i, j;
    /* vertex mapping penalty: every u of Graph 2 maps to exactly one i */
    for (u = 0; u < n; ++u) {
        int64_t s = 1;
        for (i = 0; i < n; ++i)
            s -= x[u * n + i];
        H += C1 * s * s;
    }
    /* every i of Graph 1 receives exactly one u */
    for (i = 0; i < n; ++i) {
        int64_t s = 1;
        for (u = 0; u < n; ++u)
            s -= x[u * n + i];
        H += C1 * s * s;
    }
    /* edge inconsistency: ordered (i,j) non-edge of G1 with ordered (u,v)
     * edge of G2, and ordered (i,j) edge of G1 with ordered (u,v) non-edge */
    for (i = 0; i < n; ++i)
        for (j = 0; j < n; ++j)
            for (u = 0; u < n; ++u)
                for (v = 0; v < n; ++v) {
                    int64_t xx = (int64_t)x[u * n + i] * x[v * n + j];
                    if (!xx)
                        continue;
                    if (i != j && !adj1[i * n + j] && adj2[u * n + v])
                        H += C2 * xx;
                    if (adj1[i * n + j] && u != v && !adj2[u * n + v])
                        H += C2 * xx;
                }
    return H;
}

/* Expand Eq. 8 into the upper-triangular Q of Eq. 7 plus a constant:
 * H(x) = const + sum_{a<=b} Q_ab x_a x_b, using x^2 = x. */
int or_gi_qubo(int n, const uint8_t *adj1, const uint8_t *adj2, int64_t C1,
               int64_t C2, int64_t *Q, int64_t *const_term)
{
    int N = n * n;
    int u, v, i, j, i2, u2;
    if (n < 1 || !adj1 || !adj2 || !Q || !const_term)
        return -1;
    memset(Q, 0, sizeof(int64_t) * (size_t)N * N);
    *const_term = 0;
    /* C1 (1 - sum_i x_{u,i})^2 = C1 (1 - sum_i x_{u,i} + 2 sum_{i<i2} x x) */
    for (u = 0; u < n; ++u) {
        *const_term += C1;
        for (i = 0; i < n; ++i) {
            or_q_add(Q, N, u * n + i, u * n + i, -C1);
            for (i2 = i + 1; i2 < n; ++i2)
                or_q_add(Q, N, u * n + i, u * n + i2, 2 * C1);
        }
    }
    /* C1 (1 - sum_u x_{u,i})^2, same expansion over u */
    for (i = 0; i < n; ++i) {
        *const_term += C1;
        for (u = 0; u < n; ++u) {
            or_q_add(Q, N, u * n + i, u * n + i, -C1);
            for (u2 = u + 1; u2 < n; ++u2)
                or_q_add(Q, N, u * n + i, u2 * n + i, 2 * C1);
        }
    }
    /* the two edge-inconsistency sums over ordered pairs */
    for (i = 0; i < n; ++i)
        for (j = 0; j < n; ++j)
            for (u = 0; u < n; ++u)
                for (v = 0; v < n; ++v) {
                    if (i != j && !adj1[i * n + j] && adj2[u * n + v])
                        or_q_add(Q, N, u * n + i, v * n + j, C2);
                    if (adj1[i * n + j] && u != v && !adj2[u * n + v])
                        or_q_add(Q, N, u * n + i, v * n + j, C2);
                }
    return 0;
}

/* Eq. 7 with the constant: const + sum_{a<=b} Q_ab x_a x_b. */
int64_t or_qubo_value(int N, const int64_t *Q, int64_t const_term, const uint8_t *x)
{
    int64_t H = const_term;
    int a, b;
    for (a = 0; a < N; ++a)
        for (b = a; b < N; ++b)
            H += Q[(size_t)a * N + b] * x[a] * x[b];
    return H;
}

/* QUBO -> Ising of Sec. 4.2 with sigma = 2x - 1:
 *   h_a = -Q_aa/2 - 1/4 sum_{b != a} Q_ab,   J_ab = J_ba = -Q_ab/4 (a != b),
 * where Q_ab for b < a means the stored Q_ba.  All three outputs are scaled
 * by S, which must make them integers (S divisible by 4 always does):
 *   h'[a] = S h_a, J'[a][b] = S J_ab (zero diagonal),
 *   offset' = S (const + sum_a Q_aa/2 + sum_{a<b} Q_ab/4), so that
 *   S * H_QUBO(x) = E'(sigma) + offset'. */
int or_qubo_to_ising(int N, const int64_t *Q, int64_t const_term, int64_t S,
                     int64_t *h, int64_t *J, int64_t *offset)
{
    int a, b;
    int64_t off4 = 4 * const_term; /* 4 * constant, divided at the end */
    if (N < 1 || S < 1 || !Q || !h || !J || !offset)
        return -1;
    for (a = 0; a < N; ++a) {
        int64_t h4 = -2 * Q[(size_t)a * N + a]; /* 4 * (-Q_aa / 2) */
        for (b = 0; b < N; ++b) {
            int64_t q;
            if (b == a)
                continue;
            q = a < b ? Q[(size_t)a * N + b] : Q[(size_t)b * N + a];
            h4 -= q; /* 4 * (-Q_ab / 4) */
        }
        if ((S * h4) % 4 != 0)
            return -2;
        h[a] = S * h4 / 4;
        off4 += 2 * Q[(size_t)a * N + a];
    }
    for (a = 0; a < N; ++a)
        for (b = 0; b < N; ++b) {
            int64_t q;
            if (a == b) {
                J[(size_t)a * N + b] = 0;
                continue;
            }
            q = a < b ? Q[(size_t)a * N + b] : Q[(size_t)b * N + a];
            if ((S * q) % 4 != 0)
                return -2;
            J[(size_t)a * N + b] = -S * q / 4;
            if (a < b)
                off4 += q;
        }
    if ((S * off4) % 4 != 0)
        return -2;
    *offset = S * off4 / 4;
    return 0;
}

/* Eq. 1 (and Eq. 5 per replica): H = -sum_i h_i s_i - sum_{i<j} J_ij s_i s_j. */
int64_t or_ising_energy(int N, const int64_t *h, const int64_t *J, const int8_t *s)
{
    int64_t E = 0;
    int i, j;
    for (i = 0; i < N; ++i) {
        E -= h[i] * s[i];
        for (j = i + 1; j < N; ++j)
            E -= J[(size_t)i * N + j] * s[i] * s[j];
    }
    return E;
}

void or_ising_energy_batch(int N, const int64_t *h, const int64_t *J,
                           const int8_t *s, int64_t count, int64_t *E)
{
    int64_t c;
    for (c = 0; c < count; ++c)
        E[c] = or_ising_energy(N, h, J, s + (size_t)c * N);
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  One round maps         */
/* (x0,x1,x2,x3) with round key (k0,k1) to                                    */
/*   (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)),         */
/* M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl constants  */
/* (0x9E3779B9, 0xBB67AE85) between rounds.                                   */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int r;
    for (r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The random bit of spin i, replica k, trial, cycle t (reading in header). */
int or_noise_bit(uint64_t seed, uint32_t i, uint32_t k, uint32_t trial, uint32_t t)
{
    uint32_t ctr[4], key[2], out[4], w, word, e, b;
    word = i / 32u;
    ctr[0] = 4u * (word / 16u) + word % 4u; ctr[1] = k; ctr[2] = trial; ctr[3] = t;
    key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, out);
    w = out[(word / 4u) % 4u];
    e = i % 32u;
    b = (e & 1u) ? (31u - (e >> 1)) : (15u - (e >> 1));
    return (int)((w >> b) & 1u);
}

/* ------------------------------------------------------------------------- */
/* Schedules                                                                  */
/* ------------------------------------------------------------------------- */

/* J_perp(t), Sec. 4.2 / Table 2: each iteration has tau*(beta+1) cycles; the
 * value starts at J_perp_min and grows by (J_perp_max - J_perp_min)/beta
 * every tau cycles; it is reset when a new iteration begins.  Scaled ints:
 * (jmax - jmin) must be divisible by beta. */
int32_t or_jperp(int64_t t, int32_t jmin, int32_t jmax, int32_t beta, int32_t tau)
{
    int64_t period = (int64_t)tau * (beta + 1);
    int64_t level = (t % period) / tau;
    return jmin + (int32_t)level * ((jmax - jmin) / beta);
}

/* Number of iterations of Table 2: SC / (tau (beta + 1)) with SC = EC / R. */
double or_iterations(double EC, double R, double tau, double beta)
{
    return EC / R / (tau * (beta + 1.0));
}

/* Eq. 10.  The paper notes TTS cannot be formed at P_s = 0 or 1 and that it
 * tends to 0 as P_s -> 1; the limits are returned: 0 at P_s >= 1 and
 * +infinity at P_s <= 0. */
double or_tts(double t, double p_s, double p_target)
{
    if (p_s >= 1.0)
        return 0.0;
    if (p_s <= 0.0)
        return INFINITY;
    return t * log(1.0 - p_target) / log(1.0 - p_s);
}

/* ------------------------------------------------------------------------- */
/* SSQA, Eq. 6a-6c, all N*R spins of one trial updated synchronously.         */
/* ------------------------------------------------------------------------- */
int32_t or_ssa_i0(int64_t t, int32_t i0_min, int32_t i0_max, int32_t i0_mult, int32_t tau);

typedef struct {
    int32_t N, R, cycles;
    int32_t I0, alpha, n_rnd;           /* scaled integers */
    int32_t jperp_min, jperp_max, beta, tau;
    int32_t delay;                      /* d >= 0 */
    int32_t coupling_both;              /* 0: upper replica only (Eq. 6a) */
    int32_t init_mode;                  /* 0 Philox, 1 all -1, 2 from state */
    int32_t start_cycle;                /* t of the first update */
    uint64_t seed;
    int32_t i0_max, i0_mult, i0_tau;    /* I0 schedule of Sec. 4.4; i0_max 0 = fixed I0 */
} or_params;

/* One trial.  J, h: scaled integers (J zero diagonal, symmetric).
 * State arrays are [R][N].  hist is [delay][R][N]: hist[l] = sigma(t0-1-l);
 * read when init_mode == 2, written at the end.  E_best/best_cycle track the
 * energy of sigma(t) for t = t0+1 .. t0+cycles (first cycle reaching it).
 * E_trace (optional) receives that energy every cycle, the waveform of Fig. 6:
 * E_trace[c * trace_stride + k] = E(sigma_k(t0 + c + 1)). */
int or_anneal_trial(const or_params *p, const int64_t *h, const int64_t *J,
                    uint32_t trial, int8_t *sigma, int8_t *hist, int32_t *Is,
                    int64_t *E_final, int64_t *E_best, int32_t *best_cycle,
                    int64_t *E_trace, int64_t trace_stride)
{
    int N = p->N, R = p->R, d = p->delay;
    int L = d + 1; /* levels kept: sigma(t), sigma(t-1), ..., sigma(t-d) */
    int8_t *ring, *next;
    int32_t *Is_next;
    int k, i, j, l;
    int64_t c;
    if (N < 1 || R < 1 || d < 0 || p->cycles < 0 || p->beta < 1 || p->tau < 1)
        return -1;
    ring = (int8_t *)malloc((size_t)L * R * N);
    next = (int8_t *)malloc((size_t)R * N);
    Is_next = (int32_t *)malloc(sizeof(int32_t) * (size_t)R * N);
    if (!ring || !next || !Is_next) {
        free(ring); free(next); free(Is_next);
        return -3;
    }
    /* ring[l] holds sigma(t - l) */
    if (p->init_mode == 2) {
        memcpy(ring, sigma, (size_t)R * N);
        for (l = 1; l < L; ++l)
            memcpy(ring + (size_t)l * R * N, hist + (size_t)(l - 1) * R * N, (size_t)R * N);
    } else {
        for (k = 0; k < R; ++k)
            for (i = 0; i < N; ++i) {
                int8_t s0 = -1;
                if (p->init_mode == 0)
                    s0 = or_noise_bit(p->seed, (uint32_t)i, (uint32_t)k, trial, 0xFFFFFFFFu) ? -1 : 1;
                ring[(size_t)k * N + i] = s0;
                Is[(size_t)k * N + i] = 0;
            }
        for (l = 1; l < L; ++l)
            memcpy(ring + (size_t)l * R * N, ring, (size_t)R * N);
    }
    if (E_best)
        for (k = 0; k < R; ++k) {
            E_best[k] = INT64_MAX;
            best_cycle[k] = -1;
        }

    for (c = 0; c < p->cycles; ++c) {
        int64_t t = (int64_t)p->start_cycle + c;
        int32_t jp = or_jperp(t, p->jperp_min, p->jperp_max, p->beta, p->tau);
        /* Eq. 6b uses a fixed I0 (Table 2); with an I0 schedule (SSA, Sec. 4.4)
         * the bound of cycle t is I0(t) */
        int32_t I0 = p->i0_max > p->I0 ? or_ssa_i0(t, p->I0, p->i0_max, p->i0_mult, p->i0_tau) : p->I0;
        const int8_t *cur = ring;                         /* sigma(t)     */
        const int8_t *old = ring + (size_t)d * R * N;     /* sigma(t - d) */
        for (k = 0; k < R; ++k) {
            int up = (k + 1) % R, dn = (k + R - 1) % R;
            for (i = 0; i < N; ++i) {
                int64_t F = 0, I, v;
                int32_t s_old, is_new;
                int r;
                for (j = 0; j < N; ++j)
                    F += J[(size_t)i * N + j] * cur[(size_t)k * N + j];
                r = or_noise_bit(p->seed, (uint32_t)i, (uint32_t)k, trial, (uint32_t)t) ? -1 : 1;
                /* Eq. 6a */
                I = h[i] + F + (int64_t)p->n_rnd * r + (int64_t)jp * old[(size_t)up * N + i];
                if (p->coupling_both)
                    I += (int64_t)jp * old[(size_t)dn * N + i];
                /* Eq. 6b */
                s_old = Is[(size_t)k * N + i];
                v = s_old + I;
                if (v >= I0)
                    is_new = I0 - p->alpha;
                else if (v < -I0)
                    is_new = -I0;
                else
                    is_new = (int32_t)v;
                Is_next[(size_t)k * N + i] = is_new;
                /* Eq. 6c */
                next[(size_t)k * N + i] = (int8_t)(is_new >= 0 ? 1 : -1);
            }
        }
        /* shift the history, install sigma(t+1) */
        memmove(ring + (size_t)R * N, ring, (size_t)(L - 1) * R * N);
        memcpy(ring, next, (size_t)R * N);
        memcpy(Is, Is_next, sizeof(int32_t) * (size_t)R * N);
        if (E_best || E_trace)
            for (k = 0; k < R; ++k) {
                int8_t *s = ring + (size_t)k * N;
                int64_t E = 0;
                for (i = 0; i < N; ++i) {
                    E -= h[i] * s[i];
                    for (j = i + 1; j < N; ++j)
                        E -= J[(size_t)i * N + j] * s[i] * s[j];
                }
                if (E_best && E < E_best[k]) {
                    E_best[k] = E;
                    best_cycle[k] = (int32_t)(t + 1);
                }
                if (E_trace)
                    E_trace[c * trace_stride + k] = E;
            }
    }
    memcpy(sigma, ring, (size_t)R * N);
    if (hist)
        for (l = 1; l < L; ++l)
            memcpy(hist + (size_t)(l - 1) * R * N, ring + (size_t)l * R * N, (size_t)R * N);
    if (E_final)
        for (k = 0; k < R; ++k)
            E_final[k] = or_ising_energy(N, h, J, sigma + (size_t)k * N);
    free(ring); free(next); free(Is_next);
    return 0;
}

/* All trials: trial indices trial_offset .. trial_offset + trials - 1.
 * Arrays are [trials][R][N] (hist [trials][delay][R][N]); E arrays
 * [trials][R]; E_trace [cycles][trials][R].  Optional arrays may be NULL
 * (E_best with best_cycle). */
int or_anneal(const or_params *p, const int64_t *h, const int64_t *J,
              int32_t trials, uint32_t trial_offset, int8_t *sigma, int8_t *hist,
              int32_t *Is, int64_t *E_final, int64_t *E_best, int32_t *best_cycle,
              int64_t *E_trace)
{
    size_t RN = (size_t)p->R * p->N;
    int32_t tr;
    for (tr = 0; tr < trials; ++tr) {
        int rc = or_anneal_trial(
            p, h, J, trial_offset + (uint32_t)tr, sigma + tr * RN,
            hist ? hist + (size_t)tr * p->delay * RN : NULL, Is + tr * RN,
            E_final ? E_final + (size_t)tr * p->R : NULL,
            E_best ? E_best + (size_t)tr * p->R : NULL,
            E_best ? best_cycle + (size_t)tr * p->R : NULL,
            E_trace ? E_trace + (size_t)tr * p->R : NULL, (int64_t)trials * p->R);
        if (rc)
            return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* SSA, Eq. 2a-2c, one spin network (no replicas), with the pseudo inverse   */
/* temperature schedule of Sec. 4.4: I0 starts at i0_min and is multiplied   */
/* by 1/beta (i0_mult) every tau cycles until i0_max; a new iteration starts */
/* again from i0_min.  Noise uses the SSQA bit with replica index 0.         */
/* ------------------------------------------------------------------------- */
int32_t or_ssa_i0(int64_t t, int32_t i0_min, int32_t i0_max, int32_t i0_mult, int32_t tau)
{
    int32_t levels = 1, v = i0_min, lv, l;
    while (v < i0_max) {
        v *= i0_mult;
        ++levels;
    }
    lv = (int32_t)((t % ((int64_t)tau * levels)) / tau);
    v = i0_min;
    for (l = 0; l < lv; ++l)
        v *= i0_mult;
    return v;
}

int or_ssa_trial(int N, const int64_t *h, const int64_t *J, int32_t cycles,
                 int32_t i0_min, int32_t i0_max, int32_t i0_mult, int32_t tau,
                 int32_t alpha, int32_t n_rnd, uint64_t seed, uint32_t trial,
                 int8_t *sigma, int32_t *Is)
{
    int8_t *next = (int8_t *)malloc((size_t)N);
    int32_t *Is_next = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int i, j;
    int64_t t;
    if (!next || !Is_next) {
        free(next); free(Is_next);
        return -3;
    }
    for (i = 0; i < N; ++i) {
        sigma[i] = or_noise_bit(seed, (uint32_t)i, 0u, trial, 0xFFFFFFFFu) ? -1 : 1;
        Is[i] = 0;
    }
    for (t = 0; t < cycles; ++t) {
        int32_t I0 = or_ssa_i0(t, i0_min, i0_max, i0_mult, tau);
        for (i = 0; i < N; ++i) {
            int64_t I = h[i], v;
            int r = or_noise_bit(seed, (uint32_t)i, 0u, trial, (uint32_t)t) ? -1 : 1;
            for (j = 0; j < N; ++j)
                I += J[(size_t)i * N + j] * sigma[j];
            I += (int64_t)n_rnd * r;                     /* Eq. 2a */
            v = Is[i] + I;                               /* Eq. 2b */
            Is_next[i] = v >= I0 ? I0 - alpha : (v < -I0 ? -I0 : (int32_t)v);
            next[i] = (int8_t)(Is_next[i] >= 0 ? 1 : -1); /* Eq. 2c */
        }
        memcpy(sigma, next, (size_t)N);
        memcpy(Is, Is_next, sizeof(int32_t) * (size_t)N);
    }
    free(next); free(Is_next);
    return 0;
}
