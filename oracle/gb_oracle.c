/*
 * gb_oracle.c -- plain CPU oracle for the segmented double sieve and the
 * loop-inverted Goldbach cover (GoldbachGPU, arXiv 2603.02621).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg call this file; the CUDA library never does, and this file
 * shares no code, header or table with it.
 *
 * Everything here is the plain definition written out, slowly and obviously:
 *
 *   * a prime flag is one byte per INTEGER (evens included), produced by the
 *     sieve of Eratosthenes (Sec. 2.1: the CPU baseline sieves the primes up
 *     to N first);
 *   * p_min(n) = min { p prime : n - p prime } for even n >= 4 (Sec. 2.1: the
 *     baseline walks the primes upward from 2 for each even n and tests the
 *     partner n - p; Sec. 2.3.2 names the minimal Goldbach prime and its
 *     envelope); the scan below tries p = 2, 3, 5, ... in ascending order,
 *     p <= P, and stops at the first prime whose partner is prime;
 *   * the per-segment outputs (histogram of p_min over prime index, the largest
 *     p_min with the smallest n attaining it, the count of n with no p <= P)
 *     are accumulated from those per-n values (Sec. 2.3.2 Phase 1, the
 *     unresolved counter of Sec. 2.3.2 / Phase 2 of Sec. 2.3.3);
 *   * a deterministic Miller-Rabin test for 64-bit n (Sec. 2.4) with the first
 *     twelve primes as bases (Sorenson & Webster 2015: no strong pseudoprime
 *     to all of them below 3.3e24), with exact 128-bit products;
 *   * trial division, for brute-force pins.
 *
 * Threads: segment-level parallelism with pthreads only (each thread runs the
 * same plain sequential code on its own segment).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <math.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* integer square root: largest r with r*r <= x                              */
/* ------------------------------------------------------------------------ */
uint64_t or_isqrt(uint64_t x)
{
    uint64_t r = (uint64_t)sqrtl((long double)x);
    while (r > 0 && (u128)r * r > x) r--;
    while ((u128)(r + 1) * (r + 1) <= x) r++;
    return r;
}

/* ------------------------------------------------------------------------ */
/* plain sieve of Eratosthenes on [0, x], one byte per integer               */
/* ------------------------------------------------------------------------ */
static uint8_t* plain_sieve(uint64_t x)
{
    uint8_t* f = (uint8_t*)malloc(x + 1);
    if (!f) return NULL;
    memset(f, 1, x + 1);
    f[0] = 0;
    if (x >= 1) f[1] = 0;
    for (uint64_t p = 2; p * p <= x; p++)
        if (f[p])
            for (uint64_t m = p * p; m <= x; m += p) f[m] = 0;
    return f;
}

/* small-prime cache: all primes <= small_lim, ascending */
static pthread_mutex_t g_mu = PTHREAD_MUTEX_INITIALIZER;
static uint32_t* g_small = NULL;
static uint64_t g_nsmall = 0;
static uint64_t g_small_lim = 0;

/* window flags for the integers of [a, a + len): 1 iff prime (segmented
 * Eratosthenes: every prime p <= sqrt(a + len - 1) strikes its multiples
 * m >= p*p; numbers below 2 are not prime) */
static int sieve_window_with(int64_t a, uint64_t len, uint8_t* f,
                             const uint32_t* bp, uint64_t nbp);

/* the primes <= lim, ascending, computed once and cached (grows on demand) */
static int ensure_small(uint64_t lim)
{
    pthread_mutex_lock(&g_mu);
    if (g_small_lim >= lim) { pthread_mutex_unlock(&g_mu); return 0; }
    /* grow in large steps so that nearby requests reuse one list */
    if (lim < 2 * g_small_lim) lim = 2 * g_small_lim;
    lim = (lim | ((1ull << 20) - 1));
    /* primes up to sqrt(lim) by the plain sieve, then the window sieve in
     * chunks to reach lim */
    uint64_t r = or_isqrt(lim);
    uint8_t* f = plain_sieve(r);
    if (!f) { pthread_mutex_unlock(&g_mu); return -1; }
    uint64_t nb = 0;
    for (uint64_t i = 0; i <= r; i++) nb += f[i];
    uint32_t* bp = (uint32_t*)malloc((nb + 1) * sizeof(uint32_t));
    nb = 0;
    for (uint64_t i = 0; i <= r; i++) if (f[i]) bp[nb++] = (uint32_t)i;
    free(f);
    /* upper bound on pi(lim): 1.26 lim / ln lim (Rosser-Schoenfeld), plus slack */
    double ub = lim < 100 ? 30.0 : 1.3 * (double)lim / log((double)lim) + 64.0;
    uint64_t cap = (uint64_t)ub;
    uint32_t* out = (uint32_t*)malloc(cap * sizeof(uint32_t));
    const uint64_t chunk = 1ull << 24;
    uint8_t* w = (uint8_t*)malloc(chunk);
    uint64_t n = 0;
    for (uint64_t a = 0; a <= lim; a += chunk) {
        uint64_t len = (lim + 1 - a) < chunk ? (lim + 1 - a) : chunk;
        sieve_window_with((int64_t)a, len, w, bp, nb);
        for (uint64_t i = 0; i < len; i++)
            if (w[i]) out[n++] = (uint32_t)(a + i);
    }
    free(w);
    free(bp);
    free(g_small);
    g_small = out;
    g_nsmall = n;
    g_small_lim = lim;
    pthread_mutex_unlock(&g_mu);
    return 0;
}

static int sieve_window_with(int64_t a, uint64_t len, uint8_t* f,
                             const uint32_t* bp, uint64_t nbp)
{
    memset(f, 1, len);
    int64_t end = a + (int64_t)len; /* exclusive */
    /* numbers below 2 are not prime */
    for (int64_t x = a; x < end && x < 2; x++) f[x - a] = 0;
    for (uint64_t k = 0; k < nbp; k++) {
        uint64_t p = bp[k];
        if ((int64_t)(p * p) >= end) break;
        /* first multiple of p that is >= max(a, p*p) */
        int64_t lo = a > (int64_t)(p * p) ? a : (int64_t)(p * p);
        int64_t m = (lo / (int64_t)p) * (int64_t)p;
        if (m < lo) m += (int64_t)p;
        for (; m < end; m += (int64_t)p) f[m - a] = 0;
    }
    return 0;
}

/* public: prime flags of the integers a .. a+len-1 (a may be <= 1) */
int or_sieve_window(int64_t a, uint64_t len, uint8_t* flags)
{
    if (len == 0) return 0;
    int64_t last = a + (int64_t)len - 1;
    uint64_t r = last > 0 ? or_isqrt((uint64_t)last) : 0;
    if (ensure_small(r < 16 ? 16 : r)) return -1;
    return sieve_window_with(a, len, flags, g_small, g_nsmall);
}

/* public: number of primes <= lim, and (optionally) the primes themselves */
int64_t or_primes_upto(uint64_t lim, uint32_t* out, uint64_t cap)
{
    if (ensure_small(lim < 16 ? 16 : lim)) return -1;
    uint64_t n = 0;
    for (uint64_t i = 0; i < g_nsmall && g_small[i] <= lim; i++) {
        if (out && n < cap) out[n] = g_small[i];
        n++;
    }
    return (int64_t)n;
}

/* ------------------------------------------------------------------------ */
/* p_min over a range of even n                                              */
/* ------------------------------------------------------------------------ */

/* For every even n in [lo, hi): pmin[(n - lo)/2] = the least prime p <= P such
 * that n - p is prime, or 0 if there is none.  The partner q = n - p lies in
 * [lo - P, hi), which one window sieve covers. */
static int pmin_range_with(uint64_t lo, uint64_t hi, uint32_t P, uint32_t* pmin,
                           const uint32_t* sp, uint64_t nsp, uint8_t* win)
{
    int64_t a = (int64_t)lo - (int64_t)P;
    uint64_t len = (uint64_t)((int64_t)hi - a);
    sieve_window_with(a, len, win, sp, nsp);   /* sp reaches sqrt(hi) */
    for (uint64_t n = lo; n < hi; n += 2) {
        uint32_t found = 0;
        for (uint64_t k = 0; k < nsp && sp[k] <= P; k++) {
            int64_t q = (int64_t)n - (int64_t)sp[k];
            if (q < 2) break;                 /* no prime partner below 2 */
            if (win[q - a]) { found = sp[k]; break; }
        }
        pmin[(n - lo) / 2] = found;
    }
    return 0;
}

int or_pmin_range(uint64_t lo, uint64_t hi, uint32_t P, uint32_t* pmin)
{
    if (lo & 1 || hi & 1 || lo < 4 || hi <= lo) return -1;
    uint64_t need = or_isqrt(hi) > P ? or_isqrt(hi) : P;
    if (ensure_small(need < 16 ? 16 : need)) return -1;
    uint64_t len = hi - lo + P;
    uint8_t* win = (uint8_t*)malloc(len);
    if (!win) return -1;
    int rc = pmin_range_with(lo, hi, P, pmin, g_small, g_nsmall, win);
    free(win);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* per-segment verification, threads over segments                           */
/* ------------------------------------------------------------------------ */

/* Segment k of [lo, hi) holds the even n in [lo + 2kS, min(lo + 2(k+1)S, hi)).
 * Row k of seg_out: n_checked, unresolved, max_pmin, max_pmin_n (smallest n
 * attaining the max; 0/0 when every n is unresolved).
 * Row k of seg_hist (hist_len entries): entry i counts the n whose p_min is
 * the i-th prime (p_0 = 2, p_1 = 3, ...). */
typedef struct {
    uint64_t lo, hi, S, nseg;
    uint32_t P;
    uint64_t* seg_out;
    uint64_t* seg_hist;
    uint32_t hist_len;
    uint64_t next;          /* next segment to take (under g_mu-free lock below) */
    pthread_mutex_t mu;
    const uint32_t* sp;
    uint64_t nsp;
    uint32_t* index_of;     /* prime -> its index, for p <= P */
    int err;
} verify_job;

static void* verify_worker(void* arg)
{
    verify_job* J = (verify_job*)arg;
    uint64_t S = J->S;
    uint8_t* win = (uint8_t*)malloc(2 * S + J->P + 2);
    uint32_t* pm = (uint32_t*)malloc(S * sizeof(uint32_t));
    if (!win || !pm) { J->err = -1; free(win); free(pm); return NULL; }
    for (;;) {
        pthread_mutex_lock(&J->mu);
        uint64_t k = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (k >= J->nseg) break;
        uint64_t a = J->lo + 2 * k * S;
        uint64_t b = a + 2 * S < J->hi ? a + 2 * S : J->hi;
        pmin_range_with(a, b, J->P, pm, J->sp, J->nsp, win);
        uint64_t cnt = (b - a) / 2, unres = 0, mx = 0, mxn = 0;
        uint64_t* h = J->seg_hist ? J->seg_hist + k * J->hist_len : NULL;
        if (h) memset(h, 0, J->hist_len * sizeof(uint64_t));
        for (uint64_t j = 0; j < cnt; j++) {
            uint32_t p = pm[j];
            if (p == 0) { unres++; continue; }
            if (h) {
                uint32_t idx = J->index_of[p];
                if (idx < J->hist_len) h[idx]++;
            }
            if (p > mx) { mx = p; mxn = a + 2 * j; }
        }
        uint64_t* o = J->seg_out + 4 * k;
        o[0] = cnt; o[1] = unres; o[2] = mx; o[3] = mxn;
    }
    free(win);
    free(pm);
    return NULL;
}

int or_verify_segments(uint64_t lo, uint64_t hi, uint64_t S, uint32_t P,
                       int threads, uint64_t* seg_out, uint64_t* seg_hist,
                       uint32_t hist_len)
{
    if (lo & 1 || hi & 1 || lo < 4 || hi <= lo || S == 0) return -1;
    /* the cached list must reach both P and sqrt(hi) before threads start */
    uint64_t need = or_isqrt(hi) > P ? or_isqrt(hi) : P;
    if (ensure_small(need < 16 ? 16 : need)) return -1;
    verify_job J;
    memset(&J, 0, sizeof J);
    J.lo = lo; J.hi = hi; J.S = S; J.P = P;
    J.nseg = ((hi - lo) / 2 + S - 1) / S;
    J.seg_out = seg_out; J.seg_hist = seg_hist; J.hist_len = hist_len;
    pthread_mutex_init(&J.mu, NULL);
    J.sp = g_small; J.nsp = g_nsmall;
    J.index_of = (uint32_t*)calloc((size_t)P + 1, sizeof(uint32_t));
    for (uint64_t k = 0; k < g_nsmall && g_small[k] <= P; k++)
        J.index_of[g_small[k]] = (uint32_t)k;
    if (threads < 1) threads = 1;
    pthread_t* th = (pthread_t*)malloc(threads * sizeof(pthread_t));
    for (int t = 0; t < threads; t++) pthread_create(&th[t], NULL, verify_worker, &J);
    for (int t = 0; t < threads; t++) pthread_join(th[t], NULL);
    free(th);
    free(J.index_of);
    pthread_mutex_destroy(&J.mu);
    return J.err;
}

/* ------------------------------------------------------------------------ */
/* primality of single 64-bit numbers                                         */
/* ------------------------------------------------------------------------ */

/* trial division by every integer d with d*d <= n */
int or_td_isprime(uint64_t n)
{
    if (n < 2) return 0;
    if (n < 4) return 1;
    if (n % 2 == 0) return 0;
    for (uint64_t d = 3; (u128)d * d <= n; d += 2)
        if (n % d == 0) return 0;
    return 1;
}

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((u128)a * b) % m);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}

/* Miller-Rabin with the bases 2, 3, 5, ..., 37 (the first twelve primes):
 * write n - 1 = d * 2^s with d odd; n passes base a when a^d = 1 or
 * a^(d 2^r) = n - 1 for some 0 <= r < s.  Deterministic for n < 3.3e24. */
int or_mr_isprime(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int ok = 0;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { ok = 1; break; }
        }
        if (!ok) return 0;
    }
    return 1;
}

/* p_min of one even n by ascending primes p <= P, each partner tested by
 * Miller-Rabin (Sec. 2.4, with the minimal p that Sec. 2.4 does not promise) */
uint32_t or_pmin_single(uint64_t n, uint32_t P)
{
    if (n < 4 || (n & 1)) return 0;
    if (ensure_small(P < 16 ? 16 : P)) return 0;
    for (uint64_t k = 0; k < g_nsmall && g_small[k] <= P; k++) {
        uint64_t p = g_small[k];
        if (p + 2 > n) break;
        if (or_mr_isprime(n - p)) return (uint32_t)p;
    }
    return 0;
}

/* brute force p_min by trial division of both p and n - p */
uint64_t or_td_pmin(uint64_t n)
{
    for (uint64_t p = 2; p <= n / 2; p++)
        if (or_td_isprime(p) && or_td_isprime(n - p)) return p;
    return 0;
}

/* number of Goldbach partitions c(n) = #{ p <= n/2 : p and n - p prime } */
/* ------------------------------------------------------------------------ */
/* sieve work: the strikes a segmented sieve makes in a window                 */
/* ------------------------------------------------------------------------ */
/* For the odd numbers a_odd, a_odd + 2, ..., a_odd + 2 (nbits - 1): the number
 * of pairs (p, m) with p a prime in [p_lo, p_hi], p^2 <= the window's last
 * number, and m an odd multiple of p in the window with m >= p^2 -- each
 * composite struck once per prime factor in that range, as the sieve of
 * Eratosthenes of Sec. 2.1 crosses out from p^2 on.  Counted per prime as the
 * odd j with max(p^2, a_odd) <= p j <= last. */
uint64_t or_count_strikes(int64_t a_odd, uint64_t nbits, uint64_t p_lo, uint64_t p_hi)
{
    if (nbits == 0) return 0;
    const int64_t last = a_odd + 2 * (int64_t)(nbits - 1);
    if (last < 4) return 0;
    const uint64_t r = or_isqrt((uint64_t)last);
    if (p_hi > r) p_hi = r;
    if (ensure_small(p_hi < 16 ? 16 : p_hi)) return 0;
    uint64_t total = 0;
    for (uint64_t k = 0; k < g_nsmall && g_small[k] <= p_hi; k++) {
        const uint64_t p = g_small[k];
        if (p < p_lo || p == 2) continue;
        uint64_t L = p * p;
        if (a_odd > 0 && (uint64_t)a_odd > L) L = (uint64_t)a_odd;
        const uint64_t jlo = (L + p - 1) / p, jhi = (uint64_t)last / p;
        if (jhi < jlo) continue;
        /* odd j in [jlo, jhi] */
        const uint64_t first = jlo | 1, lastj = (jhi & 1) ? jhi : jhi - 1;
        if (lastj >= first) total += (lastj - first) / 2 + 1;
    }
    return total;
}

/* number of odd t in [lo, hi] (0 if hi < lo) */
static uint64_t odd_count(uint64_t lo, uint64_t hi)
{
    if (hi < lo) return 0;
    const uint64_t first = lo | 1, last = (hi & 1) ? hi : hi - 1;
    return last >= first ? (last - first) / 2 + 1 : 0;
}

/* number of odd multiples of the odd number d in [lo, hi] */
static uint64_t odd_multiples(uint64_t lo, uint64_t hi, uint64_t d)
{
    if (hi < lo) return 0;
    return odd_count((lo + d - 1) / d, hi / d);
}

/*
 * Like or_count_strikes, counting only the multiples j*p with j coprime to 15
 * (j odd): the strikes a sieve makes when the multiples of 3 and 5 are
 * already cleared.  Per prime, by inclusion and exclusion over the odd j in
 * [jlo, jhi]: all, minus those divisible by 3, minus those divisible by 5,
 * plus those divisible by 15.
 */
uint64_t or_count_strikes_coprime15(int64_t a_odd, uint64_t nbits, uint64_t p_lo, uint64_t p_hi)
{
    if (nbits == 0) return 0;
    const int64_t last = a_odd + 2 * (int64_t)(nbits - 1);
    if (last < 4) return 0;
    const uint64_t r = or_isqrt((uint64_t)last);
    if (p_hi > r) p_hi = r;
    if (ensure_small(p_hi < 16 ? 16 : p_hi)) return 0;
    uint64_t total = 0;
    for (uint64_t k = 0; k < g_nsmall && g_small[k] <= p_hi; k++) {
        const uint64_t p = g_small[k];
        if (p < p_lo || p == 2) continue;
        uint64_t L = p * p;
        if (a_odd > 0 && (uint64_t)a_odd > L) L = (uint64_t)a_odd;
        const uint64_t jlo = (L + p - 1) / p, jhi = (uint64_t)last / p;
        if (jhi < jlo) continue;
        total += odd_multiples(jlo, jhi, 1) - odd_multiples(jlo, jhi, 3) - odd_multiples(jlo, jhi, 5) +
                 odd_multiples(jlo, jhi, 15);
    }
    return total;
}

/*
 * Like or_count_strikes_coprime15 with the multiples of 7 also left out: the
 * multiples j*p with j coprime to 105 (j odd), the strikes a sieve makes when
 * the multiples of 3, 5 and 7 are already cleared.  Per prime, by inclusion
 * and exclusion over the divisors d of 105 (sign (-1)^(number of prime
 * factors of d)) of the odd multiples of d in [jlo, jhi].
 */
uint64_t or_count_strikes_coprime105(int64_t a_odd, uint64_t nbits, uint64_t p_lo, uint64_t p_hi)
{
    if (nbits == 0) return 0;
    const int64_t last = a_odd + 2 * (int64_t)(nbits - 1);
    if (last < 4) return 0;
    const uint64_t r = or_isqrt((uint64_t)last);
    if (p_hi > r) p_hi = r;
    if (ensure_small(p_hi < 16 ? 16 : p_hi)) return 0;
    static const uint64_t div[8] = {1, 3, 5, 7, 15, 21, 35, 105};
    static const int sign[8] = {1, -1, -1, -1, 1, 1, 1, -1};
    uint64_t total = 0;
    for (uint64_t k = 0; k < g_nsmall && g_small[k] <= p_hi; k++) {
        const uint64_t p = g_small[k];
        if (p < p_lo || p == 2) continue;
        uint64_t L = p * p;
        if (a_odd > 0 && (uint64_t)a_odd > L) L = (uint64_t)a_odd;
        const uint64_t jlo = (L + p - 1) / p, jhi = (uint64_t)last / p;
        if (jhi < jlo) continue;
        int64_t c = 0;
        for (int t = 0; t < 8; t++) c += sign[t] * (int64_t)odd_multiples(jlo, jhi, div[t]);
        total += (uint64_t)c;
    }
    return total;
}

uint64_t or_partitions(uint64_t n)
{
    if (n < 4 || (n & 1)) return 0;
    uint8_t* f = (uint8_t*)malloc(n + 1);
    or_sieve_window(0, n + 1, f);
    uint64_t c = 0;
    for (uint64_t p = 2; p <= n / 2; p++)
        if (f[p] && f[n - p]) c++;
    free(f);
    return c;
}

uint64_t or_td_partitions(uint64_t n)
{
    uint64_t c = 0;
    for (uint64_t p = 2; p <= n / 2; p++)
        if (or_td_isprime(p) && or_td_isprime(n - p)) c++;
    return c;
}

/* ------------------------------------------------------------------------ */
/* prime counting, threads over chunks                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t x, chunk, nchunk, next, total;
    pthread_mutex_t mu;
} pi_job;

static void* pi_worker(void* arg)
{
    pi_job* J = (pi_job*)arg;
    uint8_t* w = (uint8_t*)malloc(J->chunk);
    for (;;) {
        pthread_mutex_lock(&J->mu);
        uint64_t c = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (c >= J->nchunk) break;
        uint64_t a = c * J->chunk;
        uint64_t len = (J->x + 1 - a) < J->chunk ? (J->x + 1 - a) : J->chunk;
        sieve_window_with((int64_t)a, len, w, g_small, g_nsmall);
        uint64_t s = 0;
        for (uint64_t i = 0; i < len; i++) s += w[i];
        pthread_mutex_lock(&J->mu);
        J->total += s;
        pthread_mutex_unlock(&J->mu);
    }
    free(w);
    return NULL;
}

/* pi(x): the number of primes <= x */
uint64_t or_prime_pi(uint64_t x, int threads)
{
    if (x < 2) return 0;
    if (ensure_small(or_isqrt(x) < 16 ? 16 : or_isqrt(x))) return 0;
    pi_job J;
    memset(&J, 0, sizeof J);
    J.x = x;
    J.chunk = 1ull << 24;
    J.nchunk = (x + 1 + J.chunk - 1) / J.chunk;
    pthread_mutex_init(&J.mu, NULL);
    if (threads < 1) threads = 1;
    pthread_t* th = (pthread_t*)malloc(threads * sizeof(pthread_t));
    for (int t = 0; t < threads; t++) pthread_create(&th[t], NULL, pi_worker, &J);
    for (int t = 0; t < threads; t++) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    return J.total;
}
