/*
 * Scalar CPU oracle for the parallel-tempering Metropolis simulation of the
 * three-dimensional +-J Edwards-Anderson model.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code with the CUDA path.
 *
 * It is deliberately plain and slow: spins are unpacked to +-1 bytes, one
 * realization and one site at a time, energies in the physical notation of
 * Eq. 1 (not the bit-sliced XOR algebra of Sec. 4.3 that the GPU uses).
 *
 *  - Hamiltonian (Sec. 2.2, Eq. 1) with h = 0:
 *        H = - sum_i sum_{d in x,y,z} J_{i,d} S_i S_{i+e_d}
 *    every nearest-neighbour bond counted once, periodic in x, y, z.
 *  - Single-spin-flip Metropolis (Sec. 2.3): flip with probability
 *    min(1, exp(-beta dE)), beta = 1/T.  The probability is an integer
 *    threshold table computed once in FP64 (Sec. 4.3.1, 4.3.2): flip iff
 *    dE <= 0 or r < metro[t][(12 - dE)/4], r a uniform 32-bit integer.
 *  - Checkerboard sweep (Sec. 3.1): all sites with (x+y+z) even, then all
 *    sites with (x+y+z) odd.
 *  - Replica exchange (Sec. 2.4, Sec. 4.1): adjacent slots p, p+1, in order
 *    p = 0..NT-2, accepted with min(1, exp((beta_p - beta_{p+1})(E_p - E_{p+1})))
 *    as the integer threshold swapt[p][k-1], k = (E_{p+1} - E_p)/4.
 *    Accepted swaps exchange the configurations between temperature slots
 *    (the paper swaps probability-table rows, Sec. 4.3.1; here each slot keeps
 *    a label of the stored configuration it currently holds).
 *  - External field (Eq. 1 with h != 0, the paper's field runs of Sec. 5):
 *        H = - sum J S S' - h sum_i S_i,  h = h_num / h_den rational,
 *    tracked exactly as Et = h_den * E_bond - h_num * M (M = sum_i S_i).  A flip
 *    of S changes Et by h_den (12 - 4u) + 2 h_num S (u = unsatisfied bonds):
 *    accepted iff that is <= 0 or r < metro_f[t][S>0][u] (a 64-bit threshold,
 *    2^32 = always).  Swaps compare Et_p - Et_{p+1}, a multiple of
 *    step = gcd(4 h_den, 2 |h_num|), with swapt[p][k-1] for Et_p - Et_{p+1} =
 *    -k step.  h_num = 0, h_den = 1 is exactly the field-free method.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11; the generator family
 *    the paper evaluates in Sec. 4.3.2), one 32-bit output per
 *    (word-group, temperature slot, copy, sweep, site), shared by the 32
 *    realizations packed in that word-group.
 *
 * Conventions fixed here (the paper leaves them open):
 *  bit 1 of a spin word  <=> S = +1;  bit 1 of a bond word <=> J = -1.
 *  site i = x + L*(y + L*z); colour(i) = (x+y+z) & 1; class index k = i >> 1.
 *  Metropolis counter  = (k >> 2, (colour << 16) | (c << 8) | t, s, g), output k & 3.
 *  Swap counter        = ((p << 3) | (b >> 2), (1 << 24) | (c << 8), P, g), output b & 3.
 *  (word 1 carries a tag in its top byte: 0 Metropolis, 1 swap).
 *  key = (seed & 0xffffffff, seed >> 32);  s = global sweep index;
 *  P = global swap-pass index.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_LANES 32

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).  Each round
 * multiplies the two even counter words by fixed odd constants, takes the
 * 64-bit products apart, and mixes the high halves with the odd words and the
 * round key; the key is bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t or_uniform(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                           int word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------ threshold tables */

/* floor(p * 2^32) clamped to the largest uint32 (Sec. 4.3.2: probabilities
 * are converted once to 32-bit unsigned integers and compared with the
 * generator's integer output). */
static uint32_t or_prob_to_u32(double p)
{
    double v = floor(ldexp(p, 32));
    if (v >= 4294967295.0) return 4294967295u;
    if (v <= 0.0) return 0u;
    return (uint32_t)v;
}

/* metro[t][u] = threshold for dE = 12 - 4u, u = 0,1,2 (the only uphill moves
 * of a site with six +-J bonds, Sec. 4.3).  Returns 0, or -1 if beta < 0. */
int or_metro_table(const double *beta, int nt, uint32_t *metro)
{
    for (int t = 0; t < nt; ++t) {
        if (!(beta[t] >= 0.0)) return -1;
        for (int u = 0; u < 3; ++u) {
            double dE = 12.0 - 4.0 * u;
            metro[t * 3 + u] = or_prob_to_u32(exp(-beta[t] * dE));
        }
    }
    return 0;
}

/* swapt[p][k-1] = threshold for E_p - E_{p+1} = -4k, k = 1..len.
 * Requires non-increasing beta (slot 0 coldest).  Returns 0 or -1. */
int or_swap_table(const double *beta, int nt, int len, uint32_t *swapt)
{
    for (int p = 0; p + 1 < nt; ++p) {
        double db = beta[p] - beta[p + 1];
        if (!(db >= 0.0)) return -1;
        for (int k = 1; k <= len; ++k)
            swapt[(size_t)p * len + (k - 1)] = or_prob_to_u32(exp(-db * 4.0 * k));
    }
    return 0;
}

/* Field tables (see the header).  metro_f[t][sp][u], sp = 1 for S = +1, is
 * floor(exp(-beta dE) 2^32) for dE = 12 - 4u + 2 h S > 0 (clamped below 2^32),
 * and 2^32 (always) for dE <= 0.  Returns 0, or -1 for beta < 0 or h_den < 1. */
int or_metro_table_field(const double *beta, int nt, int h_num, int h_den, uint64_t *metro_f)
{
    if (h_den < 1) return -1;
    const double h = (double)h_num / (double)h_den;
    for (int t = 0; t < nt; ++t) {
        if (!(beta[t] >= 0.0)) return -1;
        for (int sp = 0; sp < 2; ++sp)
            for (int u = 0; u <= 6; ++u) {
                const int S = sp ? 1 : -1;
                const long long dEt = (long long)h_den * (12 - 4 * u) + 2LL * h_num * S;
                uint64_t v = 4294967296ull;
                if (dEt > 0) v = or_prob_to_u32(exp(-beta[t] * (12.0 - 4.0 * u + 2.0 * h * S)));
                metro_f[((size_t)t * 2 + sp) * 7 + u] = v;
            }
    }
    return 0;
}

static int or_gcd(int a, int b)
{
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) { int t = a % b; a = b; b = t; }
    return a;
}

/* Step of Et differences: gcd(4 h_den, 2 |h_num|). */
int or_field_step(int h_num, int h_den) { return or_gcd(4 * h_den, 2 * h_num); }

/* swapt[p][k-1] = floor(exp(-(beta_p - beta_{p+1}) k step / h_den) 2^32), the
 * threshold for Et_p - Et_{p+1} = -k step.  Returns 0 or -1. */
int or_swap_table_field(const double *beta, int nt, int h_num, int h_den, int len, uint32_t *swapt)
{
    if (h_den < 1) return -1;
    const double step = (double)or_field_step(h_num, h_den);
    for (int p = 0; p + 1 < nt; ++p) {
        double db = beta[p] - beta[p + 1];
        if (!(db >= 0.0)) return -1;
        for (int k = 1; k <= len; ++k)
            swapt[(size_t)p * len + (k - 1)] = or_prob_to_u32(exp(-db * step * k / h_den));
    }
    return 0;
}

/* ------------------------------------------------------------ simulation */

typedef struct {
    int L, N, G, NT, C;
    uint64_t seed;
    int group_base;  /* global index of local group 0 (for runs on a subset of groups) */
    int swap_len;
    int8_t *sigma;   /* [G][C][32][NT][N]  stored configurations, +-1 */
    int8_t *J;       /* [G][32][3][N]      couplings, +-1 */
    int *nbr;        /* [N][6]  neighbour sites +x,-x,+y,-y,+z,-z (periodic) */
    int8_t *colour;  /* [N]     (x+y+z) & 1 */
    int *label;      /* [G][C][32][NT]     stored configuration held by slot t */
    int64_t *E;      /* [G][C][32][NT]     energy of stored configuration r */
    uint32_t *metro; /* [NT][3] */
    uint32_t *swapt; /* [NT-1][swap_len] */
    int h_num, h_den, step;  /* field h = h_num / h_den; step of Et differences */
    uint64_t *metro_f;       /* [NT][2][7] when h_num != 0, else NULL */
    int64_t *M;      /* [G][C][32][NT]     magnetisation of stored configuration r */
    uint64_t sweep;  /* global sweep index s of the next sweep */
    uint64_t pass;   /* global index P of the next swap pass */
} or_sim;

static int8_t *sig(const or_sim *m, int g, int c, int b, int r)
{
    return m->sigma + ((((size_t)g * m->C + c) * OR_LANES + b) * m->NT + r) * (size_t)m->N;
}
static const int8_t *jb(const or_sim *m, int g, int b, int d)
{
    return m->J + (((size_t)g * OR_LANES + b) * 3 + d) * (size_t)m->N;
}
static int *lab(const or_sim *m, int g, int c, int b)
{
    return m->label + (((size_t)g * m->C + c) * OR_LANES + b) * m->NT;
}
static int64_t *en(const or_sim *m, int g, int c, int b)
{
    return m->E + (((size_t)g * m->C + c) * OR_LANES + b) * m->NT;
}
static int64_t *mg(const or_sim *m, int g, int c, int b)
{
    return m->M + (((size_t)g * m->C + c) * OR_LANES + b) * m->NT;
}

/* Site index of (x, y, z) with periodic wrap. */
static int site(int L, int x, int y, int z)
{
    x = ((x % L) + L) % L;
    y = ((y % L) + L) % L;
    z = ((z % L) + L) % L;
    return x + L * (y + L * z);
}

/* Neighbour of site i one step along direction d (0=x,1=y,2=z), step = +-1. */
static int neighbour(int L, int i, int d, int step)
{
    int x = i % L, y = (i / L) % L, z = i / (L * L);
    if (d == 0) x += step;
    if (d == 1) y += step;
    if (d == 2) z += step;
    return site(L, x, y, z);
}

/* Eq. 1 with h = 0, each bond (i, i+e_d) once. */
static int64_t or_config_energy(const or_sim *m, const int8_t *s, int g, int b)
{
    int64_t E = 0;
    for (int i = 0; i < m->N; ++i)
        for (int d = 0; d < 3; ++d)
            E -= (int64_t)jb(m, g, b, d)[i] * s[i] * s[m->nbr[6 * i + 2 * d]];
    return E;
}

/* Local field h_i = sum over the six bonds of J_ij S_j.  The +d bond's J is
 * stored at i, the -d bond's J at the neighbour i - e_d. */
static int local_field(const or_sim *m, const int8_t *s, int g, int b, int i)
{
    int h = 0;
    for (int d = 0; d < 3; ++d) {
        int ip = m->nbr[6 * i + 2 * d];
        int im = m->nbr[6 * i + 2 * d + 1];
        h += jb(m, g, b, d)[i] * s[ip];
        h += jb(m, g, b, d)[im] * s[im];
    }
    return h;
}

static int colour_of(int L, int i)
{
    int x = i % L, y = (i / L) % L, z = i / (L * L);
    return (x + y + z) & 1;
}

void or_destroy(or_sim *m)
{
    if (!m) return;
    free(m->sigma); free(m->J); free(m->label); free(m->E); free(m->metro); free(m->swapt);
    free(m->metro_f); free(m->M);
    free(m->nbr); free(m->colour);
    free(m);
}

or_sim *or_create(int L, int G, int NT, int C, uint64_t seed,
                  const uint32_t *bonds,   /* [G][3][N] */
                  const uint32_t *spins,   /* [G][NT][C][N] */
                  const uint32_t *metro,   /* [NT][3] */
                  const uint32_t *swapt,   /* [NT-1][swap_len] */
                  int swap_len, int group_base)
{
    if (L < 2 || (L & 1) || G < 1 || NT < 1 || C < 1 || C > 2 || swap_len < 0) return NULL;
    or_sim *m = (or_sim *)calloc(1, sizeof(or_sim));
    if (!m) return NULL;
    m->L = L; m->N = L * L * L; m->G = G; m->NT = NT; m->C = C;
    m->seed = seed; m->swap_len = swap_len; m->group_base = group_base;
    size_t N = (size_t)m->N;
    m->sigma = (int8_t *)malloc((size_t)G * C * OR_LANES * NT * N);
    m->J = (int8_t *)malloc((size_t)G * OR_LANES * 3 * N);
    m->label = (int *)malloc(sizeof(int) * (size_t)G * C * OR_LANES * NT);
    m->E = (int64_t *)malloc(sizeof(int64_t) * (size_t)G * C * OR_LANES * NT);
    m->M = (int64_t *)malloc(sizeof(int64_t) * (size_t)G * C * OR_LANES * NT);
    m->h_num = 0; m->h_den = 1; m->step = 4; m->metro_f = NULL;
    m->metro = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)NT);
    m->nbr = (int *)malloc(sizeof(int) * 6 * N);
    m->colour = (int8_t *)malloc(N);
    m->swapt = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)(NT > 1 ? NT - 1 : 0) * swap_len + 1));
    if (!m->sigma || !m->J || !m->label || !m->E || !m->M || !m->metro || !m->swapt || !m->nbr ||
        !m->colour) {
        or_destroy(m);
        return NULL;
    }
    for (int i = 0; i < m->N; ++i) {
        for (int d = 0; d < 3; ++d) {
            m->nbr[6 * i + 2 * d] = neighbour(L, i, d, +1);
            m->nbr[6 * i + 2 * d + 1] = neighbour(L, i, d, -1);
        }
        m->colour[i] = (int8_t)colour_of(L, i);
    }
    memcpy(m->metro, metro, sizeof(uint32_t) * 3 * (size_t)NT);
    if (NT > 1 && swap_len > 0)
        memcpy(m->swapt, swapt, sizeof(uint32_t) * (size_t)(NT - 1) * swap_len);
    for (int g = 0; g < G; ++g)
        for (int b = 0; b < OR_LANES; ++b)
            for (int d = 0; d < 3; ++d)
                for (size_t i = 0; i < N; ++i) {
                    uint32_t w = bonds[((size_t)g * 3 + d) * N + i];
                    ((int8_t *)jb(m, g, b, d))[i] = ((w >> b) & 1u) ? -1 : +1;
                }
    for (int g = 0; g < G; ++g)
        for (int t = 0; t < NT; ++t)
            for (int c = 0; c < C; ++c)
                for (int b = 0; b < OR_LANES; ++b) {
                    int8_t *s = sig(m, g, c, b, t);
                    for (size_t i = 0; i < N; ++i) {
                        uint32_t w = spins[(((size_t)g * NT + t) * C + c) * N + i];
                        s[i] = ((w >> b) & 1u) ? +1 : -1;
                    }
                    lab(m, g, c, b)[t] = t;
                    en(m, g, c, b)[t] = or_config_energy(m, s, g, b);
                    int64_t mm = 0;
                    for (size_t i = 0; i < N; ++i) mm += s[i];
                    mg(m, g, c, b)[t] = mm;
                }
    return m;
}


/* Switches on the external field h = h_num / h_den with its Metropolis table
 * metro_f [NT][2][7] (or_metro_table_field) and the swap table given at
 * creation (built by or_swap_table_field for the same h).  Returns 0, or -1
 * for h_den < 1 or a missing table. */
int or_set_field(or_sim *m, int h_num, int h_den, const uint64_t *metro_f)
{
    if (h_den < 1 || (h_num != 0 && !metro_f)) return -1;
    m->h_num = h_num;
    m->h_den = h_den;
    /* with h_num = 0 the method is the field-free one: decisions on E, step 4 */
    m->step = h_num == 0 ? 4 : or_field_step(h_num, h_den);
    free(m->metro_f);
    m->metro_f = NULL;
    if (h_num != 0) {
        m->metro_f = (uint64_t *)malloc(sizeof(uint64_t) * 14 * (size_t)m->NT);
        if (!m->metro_f) return -1;
        memcpy(m->metro_f, metro_f, sizeof(uint64_t) * 14 * (size_t)m->NT);
    }
    return 0;
}

/* Et = h_den E - h_num M of stored configuration r. */
static int64_t et_of(const or_sim *m, int g, int c, int b, int r)
{
    return (int64_t)m->h_den * en(m, g, c, b)[r] - (int64_t)m->h_num * mg(m, g, c, b)[r];
}

/* One checkerboard sweep of the configuration held by slot t of (g, c), all
 * 32 realizations, global sweep index s (Sec. 2.3, Sec. 3.1). */
static void sweep_slot(or_sim *m, int g, int c, int t, uint64_t s)
{
    for (int colour = 0; colour < 2; ++colour) {
        for (int i = 0; i < m->N; ++i) {
            if (m->colour[i] != colour) continue;
            uint32_t k = (uint32_t)i >> 1;
            uint32_t r = or_uniform(m->seed, k >> 2,
                                    ((uint32_t)colour << 16) | ((uint32_t)c << 8) | (uint32_t)t,
                                    (uint32_t)s, (uint32_t)(m->group_base + g), (int)(k & 3u));
            for (int b = 0; b < OR_LANES; ++b) {
                int rr = lab(m, g, c, b)[t];
                int8_t *sp = sig(m, g, c, b, rr);
                int dE = 2 * sp[i] * local_field(m, sp, g, b, i);
                int accept;
                if (m->h_num == 0) {
                    if (dE <= 0) accept = 1;
                    else accept = r < m->metro[t * 3 + (12 - dE) / 4];
                } else {
                    /* Et changes by h_den dE - h_num (M' - M) = h_den dE + 2 h_num S */
                    const long long dEt = (long long)m->h_den * dE + 2LL * m->h_num * sp[i];
                    if (dEt <= 0) accept = 1;
                    else accept = (uint64_t)r < m->metro_f[((size_t)t * 2 + (sp[i] > 0)) * 7 + (12 - dE) / 4];
                }
                if (accept) {
                    mg(m, g, c, b)[rr] -= 2 * sp[i];
                    sp[i] = (int8_t)-sp[i];
                    en(m, g, c, b)[rr] += dE;
                }
            }
        }
    }
}

/* One replica-exchange pass over the slots of (g, c) with pass index P
 * (Sec. 2.4).  mask[p] receives bit b when lane b's pair (p, p+1) swapped. */
static void swap_pass(or_sim *m, int g, int c, uint64_t P, uint32_t *mask)
{
    for (int p = 0; p + 1 < m->NT; ++p) mask[p] = 0;
    for (int b = 0; b < OR_LANES; ++b) {
        int *l = lab(m, g, c, b);
        int64_t *e = en(m, g, c, b);
        for (int p = 0; p + 1 < m->NT; ++p) {
            int64_t delta = m->h_num == 0 ? e[l[p]] - e[l[p + 1]]
                                          : et_of(m, g, c, b, l[p]) - et_of(m, g, c, b, l[p + 1]);
            uint32_t r = or_uniform(m->seed, ((uint32_t)p << 3) | ((uint32_t)b >> 2),
                                    (1u << 24) | ((uint32_t)c << 8), (uint32_t)P,
                                    (uint32_t)(m->group_base + g), b & 3);
            int accept;
            if (delta >= 0) {
                accept = 1;
            } else {
                int64_t k = -delta / m->step;
                accept = (k <= m->swap_len) && (r < m->swapt[(size_t)p * m->swap_len + (k - 1)]);
            }
            if (accept) {
                int tmp = l[p]; l[p] = l[p + 1]; l[p + 1] = tmp;
                mask[p] |= 1u << b;
            }
        }
    }
}

/* Per-lane overlap count n_diff = #sites where copy 0 and copy 1 at slot t
 * disagree; the overlap is q = 1 - 2 n_diff / N. */
static int overlap_diff(const or_sim *m, int g, int t, int b)
{
    const int8_t *s0 = sig(m, g, 0, b, lab(m, g, 0, b)[t]);
    const int8_t *s1 = sig(m, g, 1, b, lab(m, g, 1, b)[t]);
    int n = 0;
    for (int i = 0; i < m->N; ++i) n += s0[i] != s1[i];
    return n;
}

typedef struct {
    or_sim *m;
    int g0, g1;
    uint64_t s0;
    int n_sweeps, swap_every;
    int32_t *energy_log;
    uint32_t *swap_log;
    uint64_t *qhist;   /* per-thread private accumulators */
    int64_t *esum;
    uint64_t measure_from;
    int measure_every;
    int check;
    int failed;
    uint64_t P0;
} or_work;

static int swap_after(uint64_t s, int swap_every)
{
    return swap_every > 0 && ((s + 1) % (uint64_t)swap_every) == 0;
}

static void *or_worker(void *arg)
{
    or_work *w = (or_work *)arg;
    or_sim *m = w->m;
    int NT = m->NT, C = m->C;
    uint32_t *mask = (uint32_t *)calloc((size_t)(NT > 1 ? NT - 1 : 1), sizeof(uint32_t));
    for (int g = w->g0; g < w->g1; ++g) {
        uint64_t P = w->P0;
        int pass_local = 0;
        for (int n = 0; n < w->n_sweeps; ++n) {
            uint64_t s = w->s0 + (uint64_t)n;
            for (int c = 0; c < C; ++c)
                for (int t = 0; t < NT; ++t) sweep_slot(m, g, c, t, s);
            if (swap_after(s, w->swap_every)) {
                for (int c = 0; c < C; ++c) {
                    swap_pass(m, g, c, P, mask);
                    if (w->swap_log)
                        for (int p = 0; p + 1 < NT; ++p)
                            w->swap_log[(((size_t)pass_local * m->G + g) * C + c) * (NT - 1) + p] = mask[p];
                }
                ++P;
                ++pass_local;
            }
            if (w->check) {
                for (int c = 0; c < C; ++c)
                    for (int b = 0; b < OR_LANES; ++b)
                        for (int r = 0; r < NT; ++r) {
                            const int8_t *sr = sig(m, g, c, b, r);
                            if (or_config_energy(m, sr, g, b) != en(m, g, c, b)[r]) w->failed = 1;
                            int64_t mm = 0;
                            for (int i = 0; i < m->N; ++i) mm += sr[i];
                            if (mm != mg(m, g, c, b)[r]) w->failed = 1;
                        }
            }
            if (w->energy_log)
                for (int t = 0; t < NT; ++t)
                    for (int c = 0; c < C; ++c)
                        for (int b = 0; b < OR_LANES; ++b)
                            w->energy_log[((((size_t)n * m->G + g) * NT + t) * C + c) * OR_LANES + b] =
                                (int32_t)en(m, g, c, b)[lab(m, g, c, b)[t]];
            int measure = s >= w->measure_from && w->measure_every > 0 &&
                          ((s - w->measure_from) % (uint64_t)w->measure_every) == 0;
            if (measure) {
                for (int t = 0; t < NT; ++t) {
                    if (w->esum)
                        for (int c = 0; c < C; ++c)
                            for (int b = 0; b < OR_LANES; ++b)
                                w->esum[t] += en(m, g, c, b)[lab(m, g, c, b)[t]];
                    if (w->qhist && C == 2)
                        for (int b = 0; b < OR_LANES; ++b)
                            w->qhist[(size_t)t * (m->N + 1) + overlap_diff(m, g, t, b)] += 1;
                }
            }
        }
    }
    free(mask);
    return NULL;
}

/* Run n_sweeps sweeps from the current global sweep index.  After sweep s a
 * swap pass runs iff swap_every > 0 and (s+1) % swap_every == 0.
 *  energy_log [n_sweeps][G][NT][C][32] int32  energies by slot at the end of each sweep
 *  swap_log   [passes][G][C][NT-1]     uint32  accepted-pair masks of each pass
 *  qhist      [NT][N+1]                uint64  += over (g, b) at measured sweeps (C == 2)
 *  esum       [NT]                     int64   += sum over (g, c, b) of E at measured sweeps
 * Sweep s is measured iff s >= measure_from and (s - measure_from) % measure_every == 0.
 * check != 0 recomputes every energy from the spins after each sweep.
 * Returns 0, or -1 when a recomputed energy differs from the tracked one. */
int or_sweep(or_sim *m, int n_sweeps, int swap_every, int32_t *energy_log, uint32_t *swap_log,
             uint64_t *qhist, int64_t *esum, uint64_t measure_from, int measure_every,
             int check, int n_threads)
{
    if (n_sweeps <= 0) return 0;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > m->G) n_threads = m->G;
    int NT = m->NT;
    or_work *w = (or_work *)calloc((size_t)n_threads, sizeof(or_work));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int j = 0; j < n_threads; ++j) {
        w[j].m = m;
        w[j].g0 = (int)((int64_t)m->G * j / n_threads);
        w[j].g1 = (int)((int64_t)m->G * (j + 1) / n_threads);
        w[j].s0 = m->sweep;
        w[j].P0 = m->pass;
        w[j].n_sweeps = n_sweeps;
        w[j].swap_every = swap_every;
        w[j].energy_log = energy_log;
        w[j].swap_log = swap_log;
        w[j].qhist = qhist ? (uint64_t *)calloc((size_t)NT * (m->N + 1), sizeof(uint64_t)) : NULL;
        w[j].esum = esum ? (int64_t *)calloc((size_t)NT, sizeof(int64_t)) : NULL;
        w[j].measure_from = measure_from;
        w[j].measure_every = measure_every;
        w[j].check = check;
    }
    if (n_threads == 1) {
        or_worker(&w[0]);
    } else {
        for (int j = 0; j < n_threads; ++j) pthread_create(&th[j], NULL, or_worker, &w[j]);
        for (int j = 0; j < n_threads; ++j) pthread_join(th[j], NULL);
    }
    int failed = 0;
    for (int j = 0; j < n_threads; ++j) {
        failed |= w[j].failed;
        if (qhist)
            for (size_t x = 0; x < (size_t)NT * (m->N + 1); ++x) qhist[x] += w[j].qhist[x];
        if (esum)
            for (int t = 0; t < NT; ++t) esum[t] += w[j].esum[t];
        free(w[j].qhist);
        free(w[j].esum);
    }
    uint64_t passes = 0;
    for (int n = 0; n < n_sweeps; ++n) passes += (uint64_t)swap_after(m->sweep + (uint64_t)n, swap_every);
    m->sweep += (uint64_t)n_sweeps;
    m->pass += passes;
    free(w);
    free(th);
    return failed ? -1 : 0;
}

/* One replica-exchange pass now, outside the sweep schedule; uses and
 * advances the global pass index.  masks [G][C][NT-1] (nullable). */
void or_pt_swap(or_sim *m, uint32_t *masks)
{
    uint32_t *mask = (uint32_t *)calloc((size_t)(m->NT > 1 ? m->NT - 1 : 1), sizeof(uint32_t));
    for (int g = 0; g < m->G; ++g)
        for (int c = 0; c < m->C; ++c) {
            swap_pass(m, g, c, m->pass, mask);
            if (masks)
                for (int p = 0; p + 1 < m->NT; ++p)
                    masks[((size_t)g * m->C + c) * (m->NT - 1) + p] = mask[p];
        }
    m->pass += 1;
    free(mask);
}

/* Tracked energies by slot: out [G][NT][C][32]. */
void or_energies(const or_sim *m, int32_t *out)
{
    for (int g = 0; g < m->G; ++g)
        for (int t = 0; t < m->NT; ++t)
            for (int c = 0; c < m->C; ++c)
                for (int b = 0; b < OR_LANES; ++b)
                    out[(((size_t)g * m->NT + t) * m->C + c) * OR_LANES + b] =
                        (int32_t)en(m, g, c, b)[lab(m, g, c, b)[t]];
}

/* Energies recomputed from the spins by Eq. 1: out [G][NT][C][32]. */
void or_energies_recompute(const or_sim *m, int32_t *out)
{
    for (int g = 0; g < m->G; ++g)
        for (int t = 0; t < m->NT; ++t)
            for (int c = 0; c < m->C; ++c)
                for (int b = 0; b < OR_LANES; ++b)
                    out[(((size_t)g * m->NT + t) * m->C + c) * OR_LANES + b] = (int32_t)
                        or_config_energy(m, sig(m, g, c, b, lab(m, g, c, b)[t]), g, b);
}

/* Magnetisations M = sum_i S_i by slot: out [G][NT][C][32]. */
void or_magnetisations(const or_sim *m, int32_t *out)
{
    for (int g = 0; g < m->G; ++g)
        for (int t = 0; t < m->NT; ++t)
            for (int c = 0; c < m->C; ++c)
                for (int b = 0; b < OR_LANES; ++b)
                    out[(((size_t)g * m->NT + t) * m->C + c) * OR_LANES + b] =
                        (int32_t)mg(m, g, c, b)[lab(m, g, c, b)[t]];
}

/* Overlap counts n_diff by slot: out [G][NT][32] (requires C == 2). */
int or_overlaps(const or_sim *m, uint32_t *out)
{
    if (m->C != 2) return -1;
    for (int g = 0; g < m->G; ++g)
        for (int t = 0; t < m->NT; ++t)
            for (int b = 0; b < OR_LANES; ++b)
                out[((size_t)g * m->NT + t) * OR_LANES + b] = (uint32_t)overlap_diff(m, g, t, b);
    return 0;
}

/* Plane counts for Fourier-mode observables (Sec. 5: the spin-glass
 * correlation length from the overlap, the ferromagnet's from the
 * magnetisation).  Site i = x + L(y + Lz); plane (axis a, index p) holds the
 * L^2 sites whose a-th coordinate is p.  mode 0: number of sites of the plane
 * where the two copies of slot t differ, out [G][NT][3][L][32] (needs C = 2);
 * mode 1: number of up spins of copy c in the plane, out [G][NT][C][3][L][32].
 * Returns 0, or -1 for an invalid mode. */
int or_plane_counts(const or_sim *m, int mode, uint32_t *out)
{
    const int L = m->L;
    if (mode == 0 && m->C != 2) return -1;
    if (mode != 0 && mode != 1) return -1;
    const int ncopy = mode == 0 ? 1 : m->C;
    for (int g = 0; g < m->G; ++g)
        for (int t = 0; t < m->NT; ++t)
            for (int c = 0; c < ncopy; ++c)
                for (int b = 0; b < OR_LANES; ++b) {
                    const int8_t *s0 = sig(m, g, c, b, lab(m, g, c, b)[t]);
                    const int8_t *s1 = mode == 0 ? sig(m, g, 1, b, lab(m, g, 1, b)[t]) : 0;
                    for (int a = 0; a < 3; ++a)
                        for (int p = 0; p < L; ++p) {
                            uint32_t n = 0;
                            for (int u = 0; u < L; ++u)
                                for (int v = 0; v < L; ++v) {
                                    const int x = a == 0 ? p : u;
                                    const int y = a == 1 ? p : (a == 0 ? u : v);
                                    const int z = a == 2 ? p : v;
                                    const int i = x + L * (y + L * z);
                                    if (mode == 0) n += s0[i] != s1[i];
                                    else n += s0[i] > 0;
                                }
                            const size_t row = mode == 0 ? (((size_t)g * m->NT + t) * 3 + a) * L + p
                                                         : ((((size_t)g * m->NT + t) * m->C + c) * 3 + a) * L + p;
                            out[row * OR_LANES + b] = n;
                        }
                }
    return 0;
}

/* Spins packed back to words, by slot: out [G][NT][C][N]. */
void or_read_spins(const or_sim *m, uint32_t *out)
{
    size_t N = (size_t)m->N;
    for (int g = 0; g < m->G; ++g)
        for (int t = 0; t < m->NT; ++t)
            for (int c = 0; c < m->C; ++c) {
                uint32_t *o = out + (((size_t)g * m->NT + t) * m->C + c) * N;
                for (size_t i = 0; i < N; ++i) o[i] = 0;
                for (int b = 0; b < OR_LANES; ++b) {
                    const int8_t *s = sig(m, g, c, b, lab(m, g, c, b)[t]);
                    for (size_t i = 0; i < N; ++i)
                        if (s[i] > 0) o[i] |= 1u << b;
                }
            }
}

uint64_t or_sweep_index(const or_sim *m) { return m->sweep; }
uint64_t or_pass_index(const or_sim *m) { return m->pass; }
