/*
 * Seeded synthetic-input generator for the SAGMS decoder workloads.
 *
 * Holds none of the decoder's arithmetic: it draws iid Z-flip error
 * patterns on n qubits and forms their syndromes s = H e (mod 2) for the
 * channel model of Sec. II (each qubit flipped independently).  Both the
 * FP64 oracle and the CUDA decoder read the bytes this file writes.
 *
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), written here from
 * its published definition: 10 rounds of two 32x32->64 multiplies with the
 * multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by the Weyl constants
 * 0x9E3779B9 / 0xBB67AE85 between rounds.
 *
 * Error positions are drawn by geometric gap sampling: with
 * T[g] = floor((1-q)^g * 2^32) (the powers formed by repeated IEEE double
 * multiplication, so every platform builds the same table), a uniform
 * u32 draw u gives a run of `g` unflipped qubits where g is the largest
 * index with u < T[g].  This is exact Bernoulli(q) sampling up to the
 * 2^-32 quantisation of the table, uses about (n*q + 1) draws per shot and
 * only integer comparisons, so x86 and Arm hosts produce identical bits.
 *
 * Layout: bit j of a pattern lives in word j/32, bit j%32 (LSB first).
 */
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

typedef struct { uint32_t v[4]; } ctr4;

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* One Philox4x32-10 block: counter c, key (k0, k1). */
void sagms_gen_philox4x32_10(const uint32_t c_in[4], const uint32_t k_in[2], uint32_t out[4]) {
    uint32_t c0 = c_in[0], c1 = c_in[1], c2 = c_in[2], c3 = c_in[3];
    uint32_t k0 = k_in[0], k1 = k_in[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (r < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Geometric-gap table for flip probability q: T[g] for g = 0..n, with T[0] = 2^32 - 1
 * standing for "always" and the table clamped at 0 once (1-q)^g * 2^32 < 1. */
static void gap_table(double q, int n, uint32_t* T) {
    double pw = 1.0;
    const double two32 = 4294967296.0;
    for (int g = 0; g <= n; ++g) {
        double t = pw * two32;
        if (g == 0 || t >= two32) T[g] = 0xFFFFFFFFu;
        else if (t < 1.0) T[g] = 0u;
        else T[g] = (uint32_t)t;
        pw *= (1.0 - q);
    }
}

/* Largest g in [0, n] with u < T[g] (T is non-increasing, T[0] = max). */
static int gap_lookup(const uint32_t* T, int n, uint32_t u) {
    if (u >= T[1 < n ? 1 : n]) return 0;
    int lo = 1, hi = n; /* invariant: u < T[lo] */
    while (lo < hi) {
        int mid = lo + (hi - lo + 1) / 2;
        if (u < T[mid]) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/*
 * Draw error patterns for shots [shot0, shot0 + shots).  q_of_shot[k] is the
 * flip probability of shot shot0 + k (0 <= q < 1).  Writes err (optional,
 * [shots][ceil(n/32)] words) and syn (optional, [shots][ceil(m/32)] words),
 * syn = H e over the CSC lists (col_ptr, row_idx) of H.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int sagms_gen_sample(int32_t m, int32_t n, const int32_t* col_ptr, const int32_t* row_idx,
                     uint64_t seed, int64_t shot0, int64_t shots, const double* q_of_shot,
                     uint32_t* err, uint32_t* syn) {
    if (m < 0 || n <= 0 || shots < 0 || !q_of_shot) return -1;
    const int nw = (n + 31) / 32, mw = (m + 31) / 32;
    uint32_t* T = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    if (!T) return -1;
    double q_cached = -1.0;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t k = 0; k < shots; ++k) {
        const double q = q_of_shot[k];
        if (!(q >= 0.0 && q < 1.0)) { free(T); return -1; }
        if (q != q_cached) { gap_table(q, n, T); q_cached = q; }
        const uint64_t shot = (uint64_t)(shot0 + k);
        uint32_t* e = err ? err + (size_t)k * nw : NULL;
        uint32_t* s = syn ? syn + (size_t)k * mw : NULL;
        if (e) memset(e, 0, sizeof(uint32_t) * nw);
        if (s) memset(s, 0, sizeof(uint32_t) * mw);
        uint32_t block[4];
        uint32_t draw = 0;
        int pos = 0;
        while (1) {
            if ((draw & 3u) == 0) {
                const uint32_t ctr[4] = {draw >> 2, (uint32_t)shot, (uint32_t)(shot >> 32), 0x53414721u};
                sagms_gen_philox4x32_10(ctr, key, block);
            }
            const uint32_t u = block[draw & 3u];
            ++draw;
            if (q == 0.0) break;
            pos += gap_lookup(T, n, u);
            if (pos >= n) break;
            if (e) e[pos >> 5] |= 1u << (pos & 31);
            if (s) {
                for (int32_t t = col_ptr[pos]; t < col_ptr[pos + 1]; ++t) {
                    const int32_t r = row_idx[t];
                    s[r >> 5] ^= 1u << (r & 31);
                }
            }
            ++pos;
            if (pos >= n) break;
        }
    }
    free(T);
    return 0;
}

/* syn = H e (mod 2) for given packed error patterns, over the CSR rows of H. */
int sagms_gen_syndrome(int32_t m, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                       int64_t shots, const uint32_t* err, uint32_t* syn) {
    if (m < 0 || n <= 0 || shots < 0 || !row_ptr || !col_idx || !err || !syn) return -1;
    const int nw = (n + 31) / 32, mw = (m + 31) / 32;
    for (int64_t k = 0; k < shots; ++k) {
        const uint32_t* e = err + (size_t)k * nw;
        uint32_t* s = syn + (size_t)k * mw;
        memset(s, 0, sizeof(uint32_t) * mw);
        for (int32_t i = 0; i < m; ++i) {
            uint32_t b = 0;
            for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
                const int32_t j = col_idx[t];
                b ^= (e[j >> 5] >> (j & 31)) & 1u;
            }
            s[i >> 5] |= b << (i & 31);
        }
    }
    return 0;
}
