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
 *
 * oracle_shadow (test acceptance only, not part of the method): replays the flooding rounds
 * of one shot with the posteriors of each check (i) taken from a supplied trace G -- the
 * posteriors another implementation reports -- and bounds, to first order in the binary32
 * unit roundoff u = 2^-24, how far that implementation's rounding may move its next
 * posteriors from the FP64 evaluation of the same step.  Round l of the replay:
 *   - decisions e_j = [sign bit of G_l(j)], residual (Eq. 1), gamma (Eq. 6), gains (Eq. 7);
 *   - CN update (Eqs. 3, 4, 8, as cn_update) on the inputs q(j,i) = G_l(j) - r(i,j), which is
 *     Eq. 2's extrinsic sum L0_j + sum_{k in N(j)\i} r(k,j) with the posterior L0_j + sum r
 *     replaced by G_l(j);
 *   - P_{l+1}(j) = L0_j + sum_{i in N(j)} r(i,j) (Eq. 2 over all edges).
 * With ORACLE_FLAG_LAYERED the checks take their inputs in layer order from the posterior as
 * it stands (G_l plus the changes of the messages already replaced that round), as the
 * layered schedule above, and the bound follows each in-place update.
 * The bound carried per edge, B(e) >= |r_impl(e) - r(e)|, grows by the rounding of each
 * binary32 step: the input difference (|q| u), the gain of Eq. 7 (a few u of its largest
 * value), the product g*min (|r| u); the minimum and the BP rule are 1-Lipschitz in their
 * inputs (for BP, d(a [+] b)/da + d(a [+] b)/db = (t_a + t_b)/(1 + t_a t_b) <= 1 with
 * t = tanh(x/2)), the BP rule adds (d_c + 6) u for its phi evaluations, and an input whose
 * sign is uncertain (|q| <= its bound) may flip the other outputs, which are then no larger
 * than that input.  The posterior bound is sum_i B(i,j) + d_v u (|L0_j| + sum_i |r(i,j)|),
 * doubled for the second-order terms the first-order analysis drops.  A trace that passes is
 * a perturbed FP64 run of the method: at every round its posteriors differ from the exact
 * step applied to its own previous state by no more than binary32 rounding can explain.
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

/* The leave-one-out set M(i)\j of edge e of check i (Eqs. 3, 4, 8): the sign parity
 * (-1)^{s_i} prod sgn(q) (1 = negative) and, over the other edges, min |q| (MS family) or
 * prod tanh(|q|/2) (BP). */
static void cn_extrinsic(int i, int e, const int32_t* row_ptr, int s_i, int msfam, const double* q, int* neg,
                         double* mn, double* prod) {
    int sg = s_i;
    double lo = INFINITY, pr = 1.0;
    for (int f = row_ptr[i]; f < row_ptr[i + 1]; ++f) {
        if (f == e) continue;
        if (q[f] < 0.0) sg ^= 1;
        const double a = fabs(q[f]);
        if (msfam) { if (a < lo) lo = a; }
        else pr *= tanh(0.5 * a);
    }
    *neg = sg;
    *mn = lo;
    *prod = pr;
}

/* The magnitude of a CN output from its leave-one-out quantities, clipped (counted in *nclip):
 * g * min (MS family, Eqs. 4, 8) or 2 atanh(prod) (BP, Eq. 3). */
static double cn_magnitude(int msfam, double g, double mn, double prod, int64_t* nclip) {
    double mag;
    if (msfam) {
        mag = g * mn;
        if (mag > MSFAM_CLIP) { mag = MSFAM_CLIP; ++*nclip; }
    } else {
        mag = (prod >= 1.0) ? INFINITY : 2.0 * atanh(prod);
        if (mag > BP_CLIP) { mag = BP_CLIP; ++*nclip; }
    }
    return mag;
}

/* (iv) for one check i: every outgoing message r(i,j) from the incoming q over M(i)\j,
 * leave-one-out written out directly (Eqs. 3, 4, 8). */
static void cn_update(int i, const int32_t* row_ptr, int s_i, int msfam, double g, const double* q, double* r,
                      int64_t* nclip) {
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int neg;
        double mn, prod;
        cn_extrinsic(i, e, row_ptr, s_i, msfam, q, &neg, &mn, &prod);
        const double mag = cn_magnitude(msfam, g, mn, prod, nclip);
        r[e] = neg ? -mag : mag;
    }
}

/* (iii) Eq. 6: the fraction of unsatisfied checks. */
static double syndrome_ratio(int unsat, int m) { return (m > 0) ? (double)unsat / (double)m : 0.0; }

/* (iii) the gain of check i: Eq. 7 for SAGMS with its residual bit, alpha for SMS, 1 for MS/BP. */
static double check_gain(int mode, double alpha, double amax, double alpha_min, double eta_unsat, double gamma,
                         int res_bit) {
    if (mode == ORACLE_MODE_SMS) return alpha;
    if (mode == ORACLE_MODE_SAGMS) return (amax - (amax - alpha_min) * gamma) * (res_bit ? eta_unsat : 1.0);
    return 1.0;
}

/* The shot's gain ceiling: Corollary 1 with Eq. 9 (alpha*(|L0|, d_c), clamped to
 * [alpha_min, 1/eta]; L0 = 0 gives alpha_min) under ORACLE_FLAG_AUTO_CEILING, else alpha_max. */
static double shot_ceiling(int auto_ceiling, double L0, int dc_max, double alpha_min, double alpha_max,
                           double eta_unsat) {
    if (!auto_ceiling) return alpha_max;
    const double x = fabs(L0);
    double a = (x > 0.0) ? oracle_alpha_star(x, dc_max) : 0.0;
    if (!(a >= alpha_min)) a = alpha_min;
    if (a > 1.0 / eta_unsat) a = 1.0 / eta_unsat;
    return a;
}

/* The prior in the units the decoder runs in (sign(L0) when normalised). */
static double prior_in_units(double l0, int normalise) {
    if (normalise) l0 = (l0 > 0.0) ? 1.0 : ((l0 < 0.0) ? -1.0 : 0.0);
    return l0;
}

/* The layered schedule's visiting order: check i goes to the smallest layer number used by no
 * check k < i sharing a qubit with it (first-fit in index order); order = checks by (layer,
 * index).  stamp needs m + 1 entries. */
static void first_fit_order(int m, const int32_t* row_ptr, const int32_t* col_idx, const int* vn_ptr,
                            const int* vn_edges, const int* edge_row, int* layer, int* order, int* stamp) {
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
    if (layered) first_fit_order(m, row_ptr, col_idx, vn_ptr, vn_edges, edge_row, layer, order, stamp);

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
        const double amax = shot_ceiling(auto_ceiling, per_qubit ? 0.0 : L0[s], dc_max, alpha_min, alpha_max, eta_unsat);
        /* prior L0_j in the units the decoder runs in */
        for (int j = 0; j < n; ++j) prior[j] = prior_in_units(per_qubit ? L0[j] : L0[s], normalise);
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
            const double gamma = syndrome_ratio(unsat, m);
            for (int i = 0; i < m; ++i) gain[i] = check_gain(mode, alpha, amax, alpha_min, eta_unsat, gamma, sres[i]);

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

/*
 * One shot's replay (see the file comment).  Arguments as oracle_decode for one shot (syn one
 * packed row, L0 one value or n values with ORACLE_FLAG_L0_PER_QUBIT), plus:
 *   rounds: rounds the implementation ran (G holds rows 0..rounds);
 *   G:      [rounds+1][n] binary32 posteriors in the units the decoder runs in;
 *   dev:    out, [rounds+1][n]: G_l(j) - P_l(j) (row 0: G_0 - L0);
 *   bnd:    out, [rounds+1][n]: the bound on |dev| (row 0: 0);
 *   flips:  out, [rounds+1]: qubits whose G_l sign bit differs from [P_l < 0].
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_shadow(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, int mode, double alpha,
                  double alpha_min, double alpha_max, double eta_unsat, unsigned flags, const uint32_t* syn,
                  const double* L0, int rounds, const float* G, double* dev, double* bnd, int32_t* flips) {
    if (m < 0 || n <= 0 || rounds < 0 || !row_ptr || !col_idx || !syn || !L0 || !G || !dev || !bnd || !flips ||
        mode < 0 || mode > 3)
        return -1;
    const double u = 0x1p-24;
    const int nnz = row_ptr[m];
    int64_t nclip = 0;
    int* vn_ptr = (int*)calloc((size_t)n + 1, sizeof(int));
    int* vn_edges = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int* fill = (int*)calloc((size_t)n + 1, sizeof(int));
    double* q = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double* bq = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double* r = (double*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
    double* br = (double*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
    double* prior = (double*)malloc(sizeof(double) * (size_t)n);
    int* sres = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    double* pc = (double*)malloc(sizeof(double) * (size_t)n);
    double* bp = (double*)malloc(sizeof(double) * (size_t)n);
    int* layer = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int* order = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int* stamp = (int*)malloc(sizeof(int) * (size_t)m + sizeof(int));
    int* edge_row = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int rc = 0;
    if (!vn_ptr || !vn_edges || !fill || !q || !bq || !r || !br || !prior || !sres || !pc || !bp || !layer ||
        !order || !stamp || !edge_row) { rc = -1; goto done; }
    for (int e = 0; e < nnz; ++e) {
        if (col_idx[e] < 0 || col_idx[e] >= n) { rc = -1; goto done; }
        vn_ptr[col_idx[e] + 1]++;
    }
    for (int j = 0; j < n; ++j) vn_ptr[j + 1] += vn_ptr[j];
    for (int e = 0; e < nnz; ++e) vn_edges[vn_ptr[col_idx[e]] + fill[col_idx[e]]++] = e;
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) edge_row[e] = i;
    {
        const int layered = (flags & ORACLE_FLAG_LAYERED) != 0;
        if (layered) first_fit_order(m, row_ptr, col_idx, vn_ptr, vn_edges, edge_row, layer, order, stamp);
        else
            for (int i = 0; i < m; ++i) order[i] = i;
        const int msfam = (mode != ORACLE_MODE_BP);
        const int per_qubit = (flags & ORACLE_FLAG_L0_PER_QUBIT) != 0;
        const int normalise = msfam && !per_qubit && !(flags & ORACLE_FLAG_NATURAL_UNITS);
        const int auto_ceiling = (flags & ORACLE_FLAG_AUTO_CEILING) && mode == ORACLE_MODE_SAGMS && !per_qubit;
        int dc_max = 0, dv_max = 0;
        for (int i = 0; i < m; ++i)
            if (row_ptr[i + 1] - row_ptr[i] > dc_max) dc_max = row_ptr[i + 1] - row_ptr[i];
        for (int j = 0; j < n; ++j)
            if (vn_ptr[j + 1] - vn_ptr[j] > dv_max) dv_max = vn_ptr[j + 1] - vn_ptr[j];
        const double amax = shot_ceiling(auto_ceiling, per_qubit ? 0.0 : L0[0], dc_max, alpha_min, alpha_max, eta_unsat);
        /* largest gain of the shot and the binary32 error of computing it (Eq. 7) */
        const double gtop = (mode == ORACLE_MODE_SAGMS) ? amax * eta_unsat : (mode == ORACLE_MODE_SMS ? alpha : 1.0);
        const double dgain = (mode == ORACLE_MODE_MS || mode == ORACLE_MODE_BP) ? 0.0
                           : (auto_ceiling ? 24.0 : 8.0) * u * gtop;
        for (int j = 0; j < n; ++j) prior[j] = prior_in_units(per_qubit ? L0[j] : L0[0], normalise);
        for (int j = 0; j < n; ++j) {
            dev[j] = (double)G[j] - prior[j];
            bnd[j] = 0.0;
        }
        {
            int f = 0;
            for (int j = 0; j < n; ++j) f += (signbit(G[j]) != 0) != (prior[j] < 0.0);
            flips[0] = f;
        }
        for (int l = 0; l < rounds; ++l) {
            const float* Gl = G + (size_t)l * n;
            /* (i) decisions of the supplied posteriors, residual (Eq. 1), gamma (Eq. 6) */
            int n_unsat = 0;
            for (int i = 0; i < m; ++i) {
                int x = bit_of(syn, i);
                for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) x ^= (signbit(Gl[col_idx[e]]) != 0);
                sres[i] = x;
                n_unsat += x;
            }
            const double gamma = syndrome_ratio(n_unsat, m);
            /* Inputs: Eq. 2's extrinsic sum with the posterior replaced by G_l.  Flooding: every
             * check takes them from G_l.  Layered: the checks in layer order take them from the
             * posterior as it stands, G_l plus the changes of the messages already replaced this
             * round (an in-place update P = (P - r_old) + r_new, rounded at each step). */
            for (int j = 0; j < n; ++j) { pc[j] = (double)Gl[j]; bp[j] = 0.0; }
            if (!layered)
                for (int e = 0; e < nnz; ++e) {
                    q[e] = pc[col_idx[e]] - r[e];
                    bq[e] = br[e] + u * (fabs(q[e]) + br[e]);
                }
            /* (iii)-(iv): gains (Eq. 7) and the CN update (Eqs. 3, 4, 8) with the bound */
            for (int o = 0; o < m; ++o) {
                const int i = order[o];
                if (layered)
                    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                        q[e] = pc[col_idx[e]] - r[e];
                        bq[e] = bp[col_idx[e]] + br[e] + u * (fabs(q[e]) + br[e]);
                    }
                const int res_i = sres[i];
                const double g = check_gain(mode, alpha, amax, alpha_min, eta_unsat, gamma, res_i);
                const int s_i = bit_of(syn, i);
                const int deg = row_ptr[i + 1] - row_ptr[i];
                for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                    int neg;
                    double mn, prod;
                    cn_extrinsic(i, e, row_ptr, s_i, msfam, q, &neg, &mn, &prod);
                    const double mag = cn_magnitude(msfam, g, mn, prod, &nclip);
                    /* bound: the largest input bound, whether an input's sign is uncertain,
                     * and (MS family) the largest bound among inputs that could be the minimum */
                    int unsure = 0;
                    double bmax = 0.0, bm = 0.0;
                    for (int f = row_ptr[i]; f < row_ptr[i + 1]; ++f)
                        if (f != e) {
                            if (fabs(q[f]) <= bq[f]) unsure = 1;
                            if (bq[f] > bmax) bmax = bq[f];
                        }
                    for (int f = row_ptr[i]; f < row_ptr[i + 1]; ++f)
                        if (f != e && fabs(q[f]) - bq[f] <= mn + bmax && bq[f] > bm) bm = bq[f];
                    double b;
                    if (msfam) {
                        b = (mn < INFINITY) ? g * bm + dgain * (mn + bm) + u * fabs(mag) : 0.0;
                        /* clipped, and every input the bound admits clips as well: exact */
                        if (mag >= MSFAM_CLIP && (g - dgain) * (mn - bm) > MSFAM_CLIP) b = 0.0;
                        if (unsure) b += 2.0 * (g + dgain) * (mn + bm);
                    } else {
                        b = bmax + (double)(deg + 6) * u + 3.0 * u * mag;
                        if (mag >= BP_CLIP) b += u * BP_CLIP;
                        if (unsure) b += 2.0 * (mag + bmax);
                    }
                    r[e] = neg ? -mag : mag;
                    br[e] = b;
                }
                if (layered)
                    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                        const int j = col_idx[e];
                        pc[j] = q[e] + r[e];
                        bp[j] = bq[e] + br[e] + u * fabs(pc[j]);
                    }
            }
            /* (v) posteriors of the replay (Eq. 2) and their bound.  A layered implementation
             * may also rebuild a posterior as the plain sum L0 + sum r (which drops its in-place
             * drift): its value must be within the bound of either form. */
            double* dl = dev + (size_t)(l + 1) * n;
            double* bl = bnd + (size_t)(l + 1) * n;
            const float* Gn = G + (size_t)(l + 1) * n;
            int f = 0;
            for (int j = 0; j < n; ++j) {
                double acc = prior[j], mag = fabs(prior[j]), bsum = 0.0;
                for (int t = vn_ptr[j]; t < vn_ptr[j + 1]; ++t) {
                    const int e = vn_edges[t];
                    acc += r[e];
                    mag += fabs(r[e]);
                    bsum += br[e];
                }
                const double bsum_fresh = 2.0 * (bsum + (double)(dv_max > 0 ? dv_max : 1) * u * mag);
                if (!layered) {
                    dl[j] = (double)Gn[j] - acc;
                    bl[j] = bsum_fresh;
                } else {
                    const double d_inplace = (double)Gn[j] - pc[j], b_inplace = 2.0 * bp[j];
                    const double d_fresh = (double)Gn[j] - acc;
                    /* report the form whose deviation is the smaller share of its bound */
                    if (fabs(d_inplace) * bsum_fresh <= fabs(d_fresh) * b_inplace) {
                        dl[j] = d_inplace; bl[j] = b_inplace; acc = pc[j];
                    } else {
                        dl[j] = d_fresh; bl[j] = bsum_fresh;
                    }
                }
                f += (signbit(Gn[j]) != 0) != (acc < 0.0);
            }
            flips[l + 1] = f;
        }
    }
done:
    free(vn_ptr); free(vn_edges); free(fill); free(q); free(bq); free(r); free(br); free(prior); free(sres);
    free(pc); free(bp); free(layer); free(order); free(stamp); free(edge_row);
    return rc;
}
