/*
 * FP64 CPU oracle for the quaternary (GF(4)) decoders of the paper: BP4 and its Min-Sum
 * family (MS, SMS, SAGMS) on a stabilizer matrix whose entries are Paulis.
 *
 * TEST INFRASTRUCTURE ONLY.  Like oracle.c this is the plain, slow statement the CUDA path
 * is checked against; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load it, and it shares no code with the CUDA library.
 *
 * Setting (Sec. II): H in GF(4)^{m x n}, entries I, X, Y, Z written here in the symplectic
 * form (x, z) of phi_s: X = (1,0) -> 1, Z = (0,1) -> 2, Y = (1,1) -> 3.  A Pauli W and an entry
 * T anticommute iff <W, T> = x_W z_T + z_W x_T = 1 (mod 2); the syndrome bit of check i is
 * s_i = sum_j <E_j, H_ij> (the trace inner product of Sec. II).  An overcomplete H (m > n - k,
 * e.g. the X- and Z-type rows of a CSS code stacked) is used as given: |S| = m.
 *
 * Messages are the scalar LLRs of the paper's equations.  Each qubit carries, per Pauli
 * W in {X, Z, Y}, the LLR Lambda_j(W) = ln P(E_j = I) / P(E_j = W); the prior is L0 =
 * ln((1 - eps0) / (eps0/3)) for every W (Sec. II), or any [n][3] table.  Readings of the
 * points the paper leaves to its reference [Lai_2021] (each also in the design notes):
 *   - VN update (Eq. 2, per Pauli): a CN message L_{k->j} counts toward Lambda(W) exactly when
 *     W anticommutes with H_kj, so Lambda_{j->i}(W) = L0_j(W) + sum_{k in N(j)\i, <W,H_kj>=1}
 *     L_{k->j}; the posterior Lambda_j(W) sums over all of N(j);
 *   - the scalar VN->CN message is the LLR that E_j commutes with T = H_ij:
 *     lambda_T = ln( (1 + e^{-Lambda(T)}) / (e^{-Lambda(T')} + e^{-Lambda(T'')}) ), with
 *     {I, T} commuting and {T', T''} anticommuting with T;  with no CN message yet this is
 *     lambda_T(L0), the first-round input (the paper's "L_{j->i}^{(1)} = L0" read per Pauli);
 *   - CN update: Eq. 3 (BP4, tanh form) or Eqs. 4 and 8 (MS family) on the scalar inputs,
 *     with the gains of Eqs. 6-7 from the residual syndrome of Eq. 1 -- the binary rules;
 *   - hard decision (Algorithm 1): e_hat_j = argmin over W in {I, X, Z, Y} of Lambda_j(W)
 *     with Lambda_j(I) = 0; ties go to the first of I, X, Z, Y;
 *   - everything in LLR units (lambda_T is not homogeneous); outputs clipped as in oracle.c
 *     (MS family 1e6, BP 23.718998); a non-finite prior marks the shot invalid.
 * Flooding schedule and stopping rule as in oracle.c: max_iter rounds, each followed by the
 * check; iters = rounds completed when the residual first vanished.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GF4_MODE_MS 0
#define GF4_MODE_SMS 1
#define GF4_MODE_SAGMS 2
#define GF4_MODE_BP 3
#define GF4_FLAG_L0_PER_QUBIT 1u
#define GF4_FLAG_NO_EARLY_STOP 2u

static const double GF4_MSFAM_CLIP = 1.0e6;
static const double GF4_BP_CLIP = 23.718998;

/* Pauli codes 1 = X, 2 = Z, 3 = Y; index into the 3-LLR arrays: X -> 0, Z -> 1, Y -> 2. */
static int anticommute(int a, int b) { return ((a & 1) & (b >> 1)) ^ ((a >> 1) & (b & 1)); }

static int gbit(const uint32_t* w, int k) { return (int)((w[k >> 5] >> (k & 31)) & 1u); }

/* ln(e^{-b} + e^{-c}), -inf-safe (b, c may be +inf). */
static double log_sum_exp_neg(double b, double c) {
    const double lo = (b < c) ? b : c, hi = (b < c) ? c : b;
    if (lo == INFINITY) return -INFINITY;
    return -lo + log1p(exp(lo - hi));
}

/* ln(1 + e^{-a}), overflow-safe. */
static double softplus_neg(double a) { return (a < 0.0 ? -a : 0.0) + log1p(exp(-fabs(a))); }

/* lambda_T of a qubit's Pauli LLRs lam[0..2] (X, Z, Y) for an entry of type T. */
static double commute_llr(const double* lam, int T) {
    const int t = (T == 1) ? 0 : (T == 2 ? 1 : 2);
    const int u = (t + 1) % 3, v = (t + 2) % 3;
    return softplus_neg(lam[t]) - log_sum_exp_neg(lam[u], lam[v]);
}

/*
 * Decode `shots` syndromes.
 *   row_ptr[m+1], col_idx[nnz], pauli[nnz] (1 X, 2 Z, 3 Y): H in CSR.
 *   syn:   [shots][ceil(m/32)] packed syndrome bits.
 *   L0:    [shots] one prior LLR per shot (the same for X, Z, Y), or with
 *          GF4_FLAG_L0_PER_QUBIT [n][3] LLRs ln P(I)/P(W), W = X, Z, Y.
 *   err:   [shots][2][ceil(n/32)] (out): the x bits, then the z bits of e_hat.
 *   conv, iters: as oracle_decode.
 *   trace: optional [shots][max_iter+1][n][3] posterior LLRs Lambda_j(X, Z, Y) at each check.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_gf4_decode(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* pauli, int mode,
                      double alpha, double alpha_min, double alpha_max, double eta_unsat, int max_iter,
                      unsigned flags, int64_t shots, const uint32_t* syn, const double* L0, uint32_t* err,
                      uint8_t* conv, int32_t* iters, double* trace) {
    if (m < 0 || n <= 0 || max_iter < 0 || shots < 0 || !row_ptr || !col_idx || !pauli || !syn || !L0 || !err ||
        !conv || !iters || mode < 0 || mode > 3)
        return -1;
    const int nnz = row_ptr[m];
    const int mw = (m + 31) / 32, nw = (n + 31) / 32;
    int* vn_ptr = (int*)calloc((size_t)n + 1, sizeof(int));
    int* vn_edges = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int* fill = (int*)calloc((size_t)n + 1, sizeof(int));
    double* lam_in = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));   /* lambda_{j->i} */
    double* r = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));        /* L_{i->j} */
    double* post = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* prior = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    int* ehat = (int*)malloc(sizeof(int) * (size_t)n);
    int* sres = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int rc = 0;
    if (!vn_ptr || !vn_edges || !fill || !lam_in || !r || !post || !prior || !ehat || !sres) { rc = -1; goto done; }
    for (int e = 0; e < nnz; ++e) {
        if (col_idx[e] < 0 || col_idx[e] >= n || pauli[e] < 1 || pauli[e] > 3) { rc = -1; goto done; }
        vn_ptr[col_idx[e] + 1]++;
    }
    for (int j = 0; j < n; ++j) vn_ptr[j + 1] += vn_ptr[j];
    for (int e = 0; e < nnz; ++e) vn_edges[vn_ptr[col_idx[e]] + fill[col_idx[e]]++] = e;
    {
        const int msfam = (mode != GF4_MODE_BP);
        const int per_qubit = (flags & GF4_FLAG_L0_PER_QUBIT) != 0;
        const int early_stop = !(flags & GF4_FLAG_NO_EARLY_STOP);
        static const int paulis[3] = {1, 2, 3};   /* X, Z, Y */
        for (int64_t s = 0; s < shots; ++s) {
            const uint32_t* sy = syn + (size_t)s * mw;
            uint32_t* ex = err + (size_t)s * 2 * nw;
            uint32_t* ez = ex + nw;
            double* tr = trace ? trace + (size_t)s * (size_t)(max_iter + 1) * (size_t)n * 3 : NULL;
            int bad = 0;
            for (int j = 0; j < n; ++j)
                for (int w = 0; w < 3; ++w) {
                    const double v = per_qubit ? L0[3 * j + w] : L0[s];
                    if (isnan(v) || v == -INFINITY) bad = 1;
                    prior[3 * j + w] = v;
                }
            if (!per_qubit && !isfinite(L0[s])) bad = 1;
            if (bad) {
                for (int k = 0; k < 2 * nw; ++k) ex[k] = 0u;
                conv[s] = 0;
                iters[s] = -1;
                continue;
            }
            for (int e = 0; e < nnz; ++e) r[e] = 0.0;
            int l = 0;
            for (;;) {
                /* (i) posterior per Pauli, decision, residual (Eq. 1) */
                for (int j = 0; j < n; ++j) {
                    double best = 0.0;
                    int arg = 0;
                    for (int w = 0; w < 3; ++w) {
                        double acc = prior[3 * j + w];
                        for (int t = vn_ptr[j]; t < vn_ptr[j + 1]; ++t) {
                            const int e = vn_edges[t];
                            if (anticommute(paulis[w], pauli[e])) acc += r[e];
                        }
                        post[3 * j + w] = acc;
                        if (acc < best) { best = acc; arg = paulis[w]; }
                    }
                    ehat[j] = arg;
                }
                if (tr) memcpy(tr + (size_t)l * n * 3, post, sizeof(double) * 3 * (size_t)n);
                int unsat = 0;
                for (int i = 0; i < m; ++i) {
                    int x = gbit(sy, i);
                    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) x ^= anticommute(ehat[col_idx[e]], pauli[e]);
                    sres[i] = x;
                    unsat += x;
                }
                /* (ii) */
                if (unsat == 0 && early_stop) { conv[s] = 1; iters[s] = l; break; }
                if (l == max_iter) { conv[s] = (unsat == 0); iters[s] = max_iter; break; }
                /* (v) of the previous round, written as the inputs of this one: the scalar
                 * VN->CN message of every edge from the extrinsic Pauli LLRs (Eq. 2 per Pauli) */
                for (int j = 0; j < n; ++j)
                    for (int t = vn_ptr[j]; t < vn_ptr[j + 1]; ++t) {
                        const int e = vn_edges[t];
                        double ext[3];
                        for (int w = 0; w < 3; ++w) {
                            double acc = prior[3 * j + w];
                            for (int u = vn_ptr[j]; u < vn_ptr[j + 1]; ++u) {
                                const int f = vn_edges[u];
                                if (f != e && anticommute(paulis[w], pauli[f])) acc += r[f];
                            }
                            ext[w] = acc;
                        }
                        lam_in[e] = commute_llr(ext, pauli[e]);
                    }
                /* (iii) gains (Eqs. 6, 7) */
                const double gamma = (m > 0) ? (double)unsat / (double)m : 0.0;
                /* (iv) CN update (Eqs. 3, 4, 8) on the scalar inputs, leave-one-out */
                for (int i = 0; i < m; ++i) {
                    double g = 1.0;
                    if (mode == GF4_MODE_SMS) g = alpha;
                    else if (mode == GF4_MODE_SAGMS) g = (alpha_max - (alpha_max - alpha_min) * gamma) * (sres[i] ? eta_unsat : 1.0);
                    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                        int neg = gbit(sy, i);
                        double mn = INFINITY, prod = 1.0;
                        for (int f = row_ptr[i]; f < row_ptr[i + 1]; ++f) {
                            if (f == e) continue;
                            if (lam_in[f] < 0.0) neg ^= 1;
                            const double a = fabs(lam_in[f]);
                            if (a < mn) mn = a;
                            prod *= tanh(0.5 * a);
                        }
                        double mag;
                        if (msfam) {
                            mag = g * mn;
                            if (mag > GF4_MSFAM_CLIP) mag = GF4_MSFAM_CLIP;
                        } else {
                            mag = (prod >= 1.0) ? INFINITY : 2.0 * atanh(prod);
                            if (mag > GF4_BP_CLIP) mag = GF4_BP_CLIP;
                        }
                        r[e] = neg ? -mag : mag;
                    }
                }
                ++l;
            }
            for (int k = 0; k < 2 * nw; ++k) ex[k] = 0u;
            for (int j = 0; j < n; ++j) {
                if (ehat[j] & 1) ex[j >> 5] |= 1u << (j & 31);
                if (ehat[j] & 2) ez[j >> 5] |= 1u << (j & 31);
            }
        }
    }
done:
    free(vn_ptr); free(vn_edges); free(fill); free(lam_in); free(r); free(post); free(prior); free(ehat); free(sres);
    return rc;
}

/*
 * oracle_gf4_shadow (test acceptance only, not part of the method): the GF(4) counterpart of
 * oracle_shadow in oracle.c.  It replays one shot's flooding rounds with the per-Pauli
 * posteriors of each check taken from a supplied binary32 trace G (another implementation's
 * Lambda(X, Z, Y) per qubit, rows 0..rounds) and bounds, to first order in u = 2^-24, how far
 * that implementation's rounding may move its next posteriors from the FP64 step.  Round l:
 *   - decisions from G_l: the argmin of (0, Lambda(X), Lambda(Z), Lambda(Y)) with the
 *     comparisons in the order X, Z, Y on the binary32 values as given, residual (Eq. 1),
 *     gamma (Eq. 6), gains (Eq. 7);
 *   - CN inputs: lambda_T(G_l(j)) - r(i,j), the extrinsic scalar message of reading 19 with
 *     the totals replaced by G_l (removing an edge's own message from the two Paulis that
 *     anticommute with its entry T subtracts it from lambda_T);
 *   - CN update (Eqs. 3, 4, 8) as in gf4_decode; Lambda_{l+1}(W) = L0 + the messages of the
 *     edges anticommuting with W (Eq. 2 per Pauli).
 * The bound per edge grows as in oracle_shadow (input difference, gain, product, 1-Lipschitz
 * minimum and BP rule, uncertain signs), with the binary32 evaluation of lambda_T adding
 * 8 u (|Lambda(T)| + |min(Lambda(T'), Lambda(T''))| + 1); lambda_T is 1-Lipschitz in the
 * largest change of its three arguments (its partial derivatives are -s(T), s(T'), s(T'') with
 * s(T) <= 1 and s(T') + s(T'') <= 1).  The posterior bound is the sum of the bounds of the
 * messages it adds plus d_v u (|L0| + their magnitudes), doubled for second-order terms.
 *   rounds, G [rounds+1][n][3] (float): as oracle_shadow; dev, bnd [rounds+1][n][3] (out):
 *   G minus the FP64 step and its bound (row 0: G_0 - L0, bound 0); flips [rounds+1] (out):
 *   qubits whose Pauli decision of G differs from that of the FP64 step.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_gf4_shadow(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* pauli,
                      int mode, double alpha, double alpha_min, double alpha_max, double eta_unsat, unsigned flags,
                      const uint32_t* syn, const double* L0, int rounds, const float* G, double* dev, double* bnd,
                      int32_t* flips) {
    if (m < 0 || n <= 0 || rounds < 0 || !row_ptr || !col_idx || !pauli || !syn || !L0 || !G || !dev || !bnd ||
        !flips || mode < 0 || mode > 3)
        return -1;
    const double u = 0x1p-24;
    const int nnz = row_ptr[m];
    int* vn_ptr = (int*)calloc((size_t)n + 1, sizeof(int));
    int* vn_edges = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int* fill = (int*)calloc((size_t)n + 1, sizeof(int));
    double* q = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double* bq = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double* r = (double*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
    double* br = (double*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
    double* prior = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    int* dec = (int*)malloc(sizeof(int) * (size_t)n);
    int* sres = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int rc = 0;
    if (!vn_ptr || !vn_edges || !fill || !q || !bq || !r || !br || !prior || !dec || !sres) { rc = -1; goto done; }
    for (int e = 0; e < nnz; ++e) {
        if (col_idx[e] < 0 || col_idx[e] >= n || pauli[e] < 1 || pauli[e] > 3) { rc = -1; goto done; }
        vn_ptr[col_idx[e] + 1]++;
    }
    for (int j = 0; j < n; ++j) vn_ptr[j + 1] += vn_ptr[j];
    for (int e = 0; e < nnz; ++e) vn_edges[vn_ptr[col_idx[e]] + fill[col_idx[e]]++] = e;
    {
        static const int paulis[3] = {1, 2, 3};   /* X, Z, Y */
        const int msfam = (mode != GF4_MODE_BP);
        const int per_qubit = (flags & GF4_FLAG_L0_PER_QUBIT) != 0;
        int dv_max = 1;
        for (int j = 0; j < n; ++j)
            if (vn_ptr[j + 1] - vn_ptr[j] > dv_max) dv_max = vn_ptr[j + 1] - vn_ptr[j];
        const double gtop = (mode == GF4_MODE_SAGMS) ? alpha_max * eta_unsat : (mode == GF4_MODE_SMS ? alpha : 1.0);
        const double dgain = (mode == GF4_MODE_MS || mode == GF4_MODE_BP) ? 0.0 : 8.0 * u * gtop;
        for (int j = 0; j < n; ++j)
            for (int w = 0; w < 3; ++w) prior[3 * j + w] = per_qubit ? L0[3 * j + w] : L0[0];
        for (int k = 0; k < 3 * n; ++k) {
            dev[k] = (double)G[k] - prior[k];
            bnd[k] = 0.0;
        }
        flips[0] = 0;
        for (int l = 0; l < rounds; ++l) {
            const float* Gl = G + (size_t)l * n * 3;
            /* (i) decisions of the supplied posteriors (their own comparisons), residual, gamma */
            for (int j = 0; j < n; ++j) {
                float best = 0.0f;
                int arg = 0;
                for (int w = 0; w < 3; ++w)
                    if (Gl[3 * j + w] < best) { best = Gl[3 * j + w]; arg = paulis[w]; }
                dec[j] = arg;
            }
            int n_unsat = 0;
            for (int i = 0; i < m; ++i) {
                int x = gbit(syn, i);
                for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) x ^= anticommute(dec[col_idx[e]], pauli[e]);
                sres[i] = x;
                n_unsat += x;
            }
            const double gamma = (m > 0) ? (double)n_unsat / (double)m : 0.0;
            /* inputs: lambda_T of the supplied totals minus the edge's own message */
            for (int e = 0; e < nnz; ++e) {
                const int j = col_idx[e], T = pauli[e];
                double lam[3];
                for (int w = 0; w < 3; ++w) lam[w] = (double)Gl[3 * j + w];
                const int t = (T == 1) ? 0 : (T == 2 ? 1 : 2);
                const double lo = (lam[(t + 1) % 3] < lam[(t + 2) % 3]) ? lam[(t + 1) % 3] : lam[(t + 2) % 3];
                const double c = commute_llr(lam, T);
                q[e] = c - r[e];
                bq[e] = br[e] + 8.0 * u * (fabs(lam[t]) + fabs(lo) + 1.0) + u * (fabs(q[e]) + br[e]);
            }
            /* CN update with the bound (as oracle_shadow) */
            for (int i = 0; i < m; ++i) {
                const int res_i = sres[i];
                double g = 1.0;
                if (mode == GF4_MODE_SMS) g = alpha;
                else if (mode == GF4_MODE_SAGMS) g = (alpha_max - (alpha_max - alpha_min) * gamma) * (res_i ? eta_unsat : 1.0);
                const int deg = row_ptr[i + 1] - row_ptr[i];
                for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                    int neg = gbit(syn, i), unsure = 0;
                    double mn = INFINITY, prod = 1.0, bmax = 0.0, bm = 0.0;
                    for (int f = row_ptr[i]; f < row_ptr[i + 1]; ++f)
                        if (f != e) {
                            if (q[f] < 0.0) neg ^= 1;
                            if (fabs(q[f]) <= bq[f]) unsure = 1;
                            if (bq[f] > bmax) bmax = bq[f];
                            if (msfam) { if (fabs(q[f]) < mn) mn = fabs(q[f]); }
                            else prod *= tanh(0.5 * fabs(q[f]));
                        }
                    double mag, b;
                    if (msfam) {
                        for (int f = row_ptr[i]; f < row_ptr[i + 1]; ++f)
                            if (f != e && fabs(q[f]) - bq[f] <= mn + bmax && bq[f] > bm) bm = bq[f];
                        mag = g * mn;
                        if (mag > GF4_MSFAM_CLIP) mag = GF4_MSFAM_CLIP;
                        b = (mn < INFINITY) ? g * bm + dgain * (mn + bm) + u * fabs(mag) : 0.0;
                        if (mag >= GF4_MSFAM_CLIP && (g - dgain) * (mn - bm) > GF4_MSFAM_CLIP) b = 0.0;
                        if (unsure) b += 2.0 * (g + dgain) * (mn + bm);
                    } else {
                        mag = (prod >= 1.0) ? INFINITY : 2.0 * atanh(prod);
                        if (mag > GF4_BP_CLIP) mag = GF4_BP_CLIP;
                        b = bmax + (double)(deg + 6) * u + 3.0 * u * mag;
                        if (mag >= GF4_BP_CLIP) b += u * GF4_BP_CLIP;
                        if (unsure) b += 2.0 * (mag + bmax);
                    }
                    r[e] = neg ? -mag : mag;
                    br[e] = b;
                }
            }
            /* (v) per-Pauli posteriors of the replay and their bound */
            double* dl = dev + (size_t)(l + 1) * n * 3;
            double* bl = bnd + (size_t)(l + 1) * n * 3;
            const float* Gn = G + (size_t)(l + 1) * n * 3;
            int fl = 0;
            for (int j = 0; j < n; ++j) {
                double sbest = 0.0;
                int sarg = 0;
                float gbest = 0.0f;
                int garg = 0;
                for (int w = 0; w < 3; ++w) {
                    double acc = prior[3 * j + w], mag = fabs(prior[3 * j + w]), bsum = 0.0;
                    for (int t2 = vn_ptr[j]; t2 < vn_ptr[j + 1]; ++t2) {
                        const int e = vn_edges[t2];
                        if (anticommute(paulis[w], pauli[e])) {
                            acc += r[e];
                            mag += fabs(r[e]);
                            bsum += br[e];
                        }
                    }
                    dl[3 * j + w] = (double)Gn[3 * j + w] - acc;
                    bl[3 * j + w] = 2.0 * (bsum + (double)dv_max * u * mag);
                    if (acc < sbest) { sbest = acc; sarg = paulis[w]; }
                    if (Gn[3 * j + w] < gbest) { gbest = Gn[3 * j + w]; garg = paulis[w]; }
                }
                fl += (sarg != garg);
            }
            flips[l + 1] = fl;
        }
    }
done:
    free(vn_ptr); free(vn_edges); free(fill); free(q); free(bq); free(r); free(br); free(prior); free(dec);
    free(sres);
    return rc;
}
