/*
 * FP64 CPU oracle for SAGMS / SMS / MS / BP syndrome decoding.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of the decoder that the CUDA path is checked against.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (paper: "Syndrome Adaptive Gain Control for Min-Sum
 * Decoding of Quantum LDPC Codes"), on a binary parity-check matrix H in CSR
 * form, for each shot:
 *
 *   State: one double per Tanner-graph edge e = (i, j) for the VN->CN message
 *   q[e] = L_{j->i} and one for the CN->VN message r[e] = L_{i->j}.
 *   Init (Sec. II, BP4 decoder): q[e] = L0_j, r[e] = 0.
 *   For l = 1, 2, ... (Algorithm 1):
 *     (i)   posterior P_j = L0_j + sum_{i in N(j)} r(i,j); hard decision
 *           e_hat_j = [P_j < 0]; residual syndrome s~ = s XOR H e_hat (Eq. 1);
 *     (ii)  s~ = 0 -> success, iters = l - 1 (rounds completed);
 *           after max_iter rounds -> failure, iters = max_iter;
 *     (iii) syndrome ratio gamma = |s~|_0 / m (Eq. 6) and per-check gain
 *           g_i (Eq. 7 for SAGMS; alpha for SMS; 1 for MS);
 *     (iv)  CN update for every edge, as the leave-one-out over M(i)\j written
 *           out directly:
 *             MS family (Eqs. 4, 8): r = (-1)^{s_i} prod sgn(q) * g_i * min |q|
 *             BP (Eq. 3, tanh form): r = (-1)^{s_i} prod sgn(q) * 2 atanh(prod tanh(|q|/2))
 *           (the tanh product is the same function as phi^{-1}(sum phi) with
 *           phi(x) = -log tanh(x/2), evaluated in the product domain);
 *     (v)   VN update for every edge (Eq. 2): q(j,i) = L0_j + sum_{k in N(j)\i} r(k,j),
 *           again as a direct leave-one-out sum, using the CN messages of (iv).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   - binary hard decision: e_hat_j = 1 iff P_j < 0 (P_j = 0 -> 0);
 *     sgn(0) = +1 in the sign products;
 *   - s~_i in Eq. 7 is the residual bit; (-1)^{s_i} in Eqs. 3/4/8 uses the
 *     input syndrome bit; |S| = m (rows of the supplied H);
 *   - flooding schedule: (v) uses the CN messages just computed in (iv);
 *   - max_iter message-passing rounds, each followed by the (i)/(ii) check;
 *   - MS family with a per-shot scalar L0 runs in L0-normalised units (every
 *     message divided by |L0|, prior sign(L0)): the MS/SMS/SAGMS updates are
 *     positively homogeneous of degree 1, so this changes no decision and
 *     makes MS exact-integer (ties resolve identically in any precision);
 *   - MS-family CN outputs are clipped to |r| <= 1e6 (normalised units when
 *     normalised), BP outputs to |r| <= 23.718998 = ln(2e10), the cap implied
 *     by the 1e-10 guard of the paper's BP transfer-function plot (Fig. 1b);
 *   - degree-1 checks: the leave-one-out set is empty, so min = +inf
 *     (MS family) or prod = 1 (BP) and the output saturates at the clip;
 *   - input validation (not part of the method): a non-finite prior marks the
 *     shot invalid (e_hat = 0, conv = 0, iters = -1);
 *   - ORACLE_FLAG_AUTO_CEILING (SAGMS, per-shot prior): the gain ceiling of
 *     Corollary 1, alpha_max = alpha*(|L0|, d_c) of Eq. 9 per shot with d_c the
 *     largest check degree, clamped to [alpha_min, 1/eta]; L0 = 0 gives alpha_min.
 *
 * ORACLE_FLAG_LAYERED: a layered (serial-check) schedule, which the paper does not
 * use; it replaces (iv) and (v) of each round, everything else staying as above:
 *   - layers: check i goes to the smallest layer number used by no check k < i that
 *     shares a qubit with it (first-fit colouring of the checks in index order), so
 *     the checks of one layer share no qubit;
 *   - a round visits the layers in increasing order and, in each, every check i
 *     (index order; checks of a layer commute): first its inputs
 *     q(j,i) = L0_j + sum_{k in N(j)\i} r(k,j) from the CN messages as they stand
 *     (Eq. 2, including those already replaced earlier in the round), then its
 *     outputs r(i,j) by the rule of (iv) with the round's gain g_i;
 *   - the gains of a round come from the residual at its start, (i)-(iii), as in
 *     the flooding schedule.
 *
 * ORACLE_FLAG_PERTURB (test acceptance only, not part of the method): a model of FP32
 * rounding for the conditioning analysis of the GPU tests.  Every posterior of (i) and every
 * VN->CN input of (v) or of a layered round is moved by s * 2^-23 * (|L0_j| + the sum of the
 * magnitudes of its terms), with s = +-1 a fixed pseudo-random sign per item and round
 * (the splitmix64 finaliser of Steele, Lea and Flood, OOPSLA 2014, on the item and round
 * numbers), all signs flipped under ORACLE_FLAG_PERTURB_NEG.  A shot whose outcome moves
 * under it has no answer that FP32 arithmetic determines.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MODE_MS 0
#define ORACLE_MODE_SMS 1
#define ORACLE_MODE_SAGMS 2
#define ORACLE_MODE_BP 3

#define ORACLE_FLAG_L0_PER_QUBIT 1u
#define ORACLE_FLAG_NO_EARLY_STOP 2u
#define ORACLE_FLAG_NATURAL_UNITS 8u  /* oracle only: keep the MS family in LLR units */
#define ORACLE_FLAG_AUTO_CEILING 16u
#define ORACLE_FLAG_LAYERED 32u
#define ORACLE_FLAG_PERTURB 64u       /* test only: the FP32 rounding model below */
#define ORACLE_FLAG_PERTURB_NEG 128u  /* test only: its mirror image */

double oracle_alpha_star(double L0, int dc);

static const double MSFAM_CLIP = 1.0e6;
static const double BP_CLIP = 23.718998;

static int bit_of(const uint32_t* w, int k) { return (int)((w[k >> 5] >> (k & 31)) & 1u); }

/* +1 or -1, a fixed function of (item, round) (ORACLE_FLAG_PERTURB). */
static double pert_sign(uint64_t item, uint64_t round) {
    uint64_t z = item * 0x9E3779B97F4A7C15ull + (round + 1u) * 0xD1B54A32D192ED03ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (z & 1u) ? 1.0 : -1.0;
}

/* (iv) for one check i: every outgoing message r(i,j) from the incoming q over M(i)\j,
 * leave-one-out written out directly (Eqs. 3, 4, 8). */
static void cn_update(int i, const int32_t* row_ptr, int s_i, int msfam, double g, const double* q, double* r,
                      int64_t* nclip) {
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int neg = s_i;
        double mn = INFINITY, prod = 1.0;
        for (int f = row_ptr[i]; f < row_ptr[i + 1]; ++f) {
            if (f == e) continue;
            if (q[f] < 0.0) neg ^= 1;
            const double a = fabs(q[f]);
            if (msfam) { if (a < mn) mn = a; }
            else prod *= tanh(0.5 * a);
        }
        double mag;
        if (msfam) {
            mag = g * mn;
            if (mag > MSFAM_CLIP) { mag = MSFAM_CLIP; ++*nclip; }
        } else {
            mag = (prod >= 1.0) ? INFINITY : 2.0 * atanh(prod);
            if (mag > BP_CLIP) { mag = BP_CLIP; ++*nclip; }
        }
        r[e] = neg ? -mag : mag;
    }
}

/*
 * Decode `shots` syndromes.
 *   row_ptr[m+1], col_idx[nnz]: H in CSR (any column order, no duplicates).
 *   syn:   [shots][ceil(m/32)] packed input syndromes.
 *   L0:    [shots] (per-shot scalar prior) or, with ORACLE_FLAG_L0_PER_QUBIT, [n].
 *   err:   [shots][ceil(n/32)] packed e_hat (out).
 *   conv:  [shots] 1 if s~ = 0 at return (out).   iters: [shots] (out).
 *   trace: optional [shots][max_iter+1][n] posteriors P_j at each check (i),
 *          in the units the decoder runs in; rows after the return are left as is.
 *   scale: optional, same layout: |L0_j| + sum_{i in N(j)} |r(i,j)| at each check (i), the
 *          magnitude of the terms of P_j's sum, which bounds the rounding error a
 *          lower-precision evaluation of P_j carries (test acceptance; not part of the method).
 *   clips: optional [shots] (out): CN outputs of the shot that the clip bound.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_decode(int m, int n, const int32_t* row_ptr, const int32_t* col_idx,
                  int mode, double alpha, double alpha_min, double alpha_max, double eta_unsat,
                  int max_iter, unsigned flags, int64_t shots,
                  const uint32_t* syn, const double* L0,
                  uint32_t* err, uint8_t* conv, int32_t* iters, double* trace, double* scale, int64_t* clips) {
    if (m < 0 || n <= 0 || max_iter < 0 || shots < 0 || !row_ptr || !col_idx || !syn || !L0 ||
        !err || !conv || !iters || mode < 0 || mode > 3)
        return -1;
    const int nnz = row_ptr[m];
    const int mw = (m + 31) / 32, nw = (n + 31) / 32;

    /* CSC edge lists: for VN j, the edge ids e (positions in col_idx) of its checks. */
    int* vn_ptr = (int*)calloc((size_t)n + 1, sizeof(int));
    int* vn_edges = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int* edge_row = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double* r = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double* P = (double*)malloc(sizeof(double) * (size_t)n);
    double* prior = (double*)malloc(sizeof(double) * (size_t)n);
    double* gain = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int* ehat = (int*)malloc(sizeof(int) * (size_t)n);
    int* sres = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int* fill = (int*)calloc((size_t)n + 1, sizeof(int));
    int* layer = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int* order = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int* stamp = (int*)malloc(sizeof(int) * (size_t)m + sizeof(int));
    int rc = 0;
    if (!vn_ptr || !vn_edges || !edge_row || !q || !r || !P || !prior || !gain || !ehat || !sres || !fill ||
        !layer || !order || !stamp) {
        rc = -1;
        goto done;
    }
    for (int i = 0; i < m; ++i) {
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int j = col_idx[e];
            if (j < 0 || j >= n) { rc = -1; goto done; }
            edge_row[e] = i;
            vn_ptr[j + 1]++;
        }
    }
    for (int j = 0; j < n; ++j) vn_ptr[j + 1] += vn_ptr[j];
    for (int e = 0; e < nnz; ++e) {
        const int j = col_idx[e];
        vn_edges[vn_ptr[j] + fill[j]++] = e;
    }

    const int msfam = (mode != ORACLE_MODE_BP);
    const int per_qubit = (flags & ORACLE_FLAG_L0_PER_QUBIT) != 0;
    const int auto_ceiling = (flags & ORACLE_FLAG_AUTO_CEILING) && mode == ORACLE_MODE_SAGMS && !per_qubit;
    int dc_max = 0;
    for (int i = 0; i < m; ++i)
        if (row_ptr[i + 1] - row_ptr[i] > dc_max) dc_max = row_ptr[i + 1] - row_ptr[i];
    const int normalise = msfam && !per_qubit && !(flags & ORACLE_FLAG_NATURAL_UNITS);
    const int early_stop = !(flags & ORACLE_FLAG_NO_EARLY_STOP);
    const int layered = (flags & ORACLE_FLAG_LAYERED) != 0;
    const double pert = (flags & ORACLE_FLAG_PERTURB) ? ((flags & ORACLE_FLAG_PERTURB_NEG) ? -0x1p-23 : 0x1p-23) : 0.0;
    if (layered) {
        /* first-fit layer of every check in index order, then the checks by (layer, index) */
        int nlayers = 0;
        for (int i = 0; i < m; ++i) {
            for (int k = 0; k <= m; ++k) stamp[k] = 0;
            for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                const int j = col_idx[e];
                for (int u = vn_ptr[j]; u < vn_ptr[j + 1]; ++u) {
                    const int k = edge_row[vn_edges[u]];
                    if (k < i) stamp[layer[k]] = 1;
                }
            }
            int l = 0;
            while (stamp[l]) ++l;
            layer[i] = l;
            if (l + 1 > nlayers) nlayers = l + 1;
        }
        int o = 0;
        for (int l = 0; l < nlayers; ++l)
            for (int i = 0; i < m; ++i)
                if (layer[i] == l) order[o++] = i;
    }

    for (int64_t s = 0; s < shots; ++s) {
        const uint32_t* sy = syn + (size_t)s * mw;
        uint32_t* eo = err + (size_t)s * nw;
        double* tr = trace ? trace + (size_t)s * (size_t)(max_iter + 1) * (size_t)n : NULL;
        double* sc = scale ? scale + (size_t)s * (size_t)(max_iter + 1) * (size_t)n : NULL;
        int64_t nclip = 0;

        /* A non-finite prior marks the shot invalid: e_hat = 0, conv = 0, iters = -1. */
        int bad = 0;
        for (int j = 0; j < (per_qubit ? n : 1); ++j)
            if (!isfinite(per_qubit ? L0[j] : L0[s])) bad = 1;
        if (bad) {
            for (int k = 0; k < nw; ++k) eo[k] = 0u;
            conv[s] = 0;
            iters[s] = -1;
            continue;
        }
        /* the shot's gain ceiling (Corollary 1 with Eq. 9), or the alpha_max parameter */
        double amax = alpha_max;
        if (auto_ceiling) {
            const double x = fabs(L0[s]);
            double a = (x > 0.0) ? oracle_alpha_star(x, dc_max) : 0.0;
            if (!(a >= alpha_min)) a = alpha_min;
            if (a > 1.0 / eta_unsat) a = 1.0 / eta_unsat;
            amax = a;
        }
        /* prior L0_j in the units the decoder runs in */
        for (int j = 0; j < n; ++j) {
            double l0 = per_qubit ? L0[j] : L0[s];
            if (normalise) l0 = (l0 > 0.0) ? 1.0 : ((l0 < 0.0) ? -1.0 : 0.0);
            prior[j] = l0;
        }
        /* Init (Sec. II): L_{j->i} = L0, CN->VN messages zero. */
        for (int e = 0; e < nnz; ++e) { q[e] = prior[col_idx[e]]; r[e] = 0.0; }

        int l = 0;
        for (;;) {
            /* (i) posterior, hard decision, residual syndrome (Eq. 1) */
            for (int j = 0; j < n; ++j) {
                double acc = prior[j], mag = fabs(prior[j]);
                for (int t = vn_ptr[j]; t < vn_ptr[j + 1]; ++t) {
                    acc += r[vn_edges[t]];
                    mag += fabs(r[vn_edges[t]]);
                }
                if (pert != 0.0) acc += pert * pert_sign((uint64_t)nnz + (uint64_t)j, (uint64_t)l) * mag;
                P[j] = acc;
                ehat[j] = (acc < 0.0) ? 1 : 0;
            }
            if (tr) memcpy(tr + (size_t)l * n, P, sizeof(double) * (size_t)n);
            if (sc) {
                for (int j = 0; j < n; ++j) {
                    double a = fabs(prior[j]);
                    for (int t = vn_ptr[j]; t < vn_ptr[j + 1]; ++t) a += fabs(r[vn_edges[t]]);
                    sc[(size_t)l * n + j] = a;
                }
            }
            int unsat = 0;
            for (int i = 0; i < m; ++i) {
                int x = bit_of(sy, i);
                for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) x ^= ehat[col_idx[e]];
                sres[i] = x;
                unsat += x;
            }
            /* (ii) early termination / iteration budget */
            if (unsat == 0 && early_stop) { conv[s] = 1; iters[s] = l; break; }
            if (l == max_iter) { conv[s] = (unsat == 0); iters[s] = max_iter; break; }

            /* (iii) syndrome ratio (Eq. 6) and per-CN gain (Eq. 7) */
            const double gamma = (m > 0) ? (double)unsat / (double)m : 0.0;
            for (int i = 0; i < m; ++i) {
                if (mode == ORACLE_MODE_MS) gain[i] = 1.0;
                else if (mode == ORACLE_MODE_SMS) gain[i] = alpha;
                else if (mode == ORACLE_MODE_SAGMS)
                    gain[i] = (amax - (amax - alpha_min) * gamma) * (sres[i] ? eta_unsat : 1.0);
                else gain[i] = 1.0;
            }

            if (!layered) {
                /* (iv) CN update of every check (Eqs. 3, 4, 8) */
                for (int i = 0; i < m; ++i) cn_update(i, row_ptr, bit_of(sy, i), msfam, gain[i], q, r, &nclip);
                /* (v) VN update, leave-one-out over N(j)\i (Eq. 2) */
                for (int j = 0; j < n; ++j) {
                    for (int t = vn_ptr[j]; t < vn_ptr[j + 1]; ++t) {
                        const int e = vn_edges[t];
                        double acc = prior[j], mag = fabs(prior[j]);
                        for (int u = vn_ptr[j]; u < vn_ptr[j + 1]; ++u)
                            if (u != t) {
                                acc += r[vn_edges[u]];
                                mag += fabs(r[vn_edges[u]]);
                            }
                        if (pert != 0.0) acc += pert * pert_sign((uint64_t)e, (uint64_t)l) * mag;
                        q[e] = acc;
                    }
                }
            } else {
                /* layered round: each check in layer order takes its inputs from the CN
                 * messages as they stand (Eq. 2), then updates its outputs */
                for (int o = 0; o < m; ++o) {
                    const int i = order[o];
                    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                        const int j = col_idx[e];
                        double acc = prior[j], mag = fabs(prior[j]);
                        for (int u = vn_ptr[j]; u < vn_ptr[j + 1]; ++u)
                            if (vn_edges[u] != e) {
                                acc += r[vn_edges[u]];
                                mag += fabs(r[vn_edges[u]]);
                            }
                        if (pert != 0.0) acc += pert * pert_sign((uint64_t)e, (uint64_t)l) * mag;
                        q[e] = acc;
                    }
                    cn_update(i, row_ptr, bit_of(sy, i), msfam, gain[i], q, r, &nclip);
                }
            }
            ++l;
        }
        for (int k = 0; k < nw; ++k) eo[k] = 0u;
        for (int j = 0; j < n; ++j)
            if (ehat[j]) eo[j >> 5] |= 1u << (j & 31);
        if (clips) clips[s] = nclip;
    }

done:
    free(vn_ptr); free(vn_edges); free(edge_row); free(q); free(r); free(P); free(prior);
    free(gain); free(ehat); free(sres); free(fill); free(layer); free(order); free(stamp);
    return rc;
}

/* Closed form of Eq. 9: alpha*(L0, dc) = 2 atanh(tanh(L0/2)^(dc-1)) / L0. */
double oracle_alpha_star(double L0, int dc) {
    return 2.0 * atanh(pow(tanh(0.5 * L0), (double)(dc - 1))) / L0;
}

/* First-order form of Eq. 9: 1 - ln(dc - 1) / L0. */
double oracle_alpha_star_approx(double L0, int dc) {
    return 1.0 - log((double)(dc - 1)) / L0;
}
