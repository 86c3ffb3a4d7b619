// libsagms.so: C ABI (include/sagms.h) around the batched decoder kernels.
//
// Host responsibilities: validate the CSR matrix and the parameters; at load time, fix the
// edge order every layout shares (column-indexed slots by edge colouring where needed) and
// lay the Tanner graph out once per kernel that covers the code (slot-major index arrays,
// two-slot and two-group offsets, column-indexed offsets, layered-schedule records); at
// decode time, pick the kernel and grid and launch on the caller's stream.  Every step of
// the decode itself runs in the kernels: decode_qc.cuh, decode_groups.cuh,
// decode_slots.cuh and decode_kernel.cuh (flooding schedule) and decode_layered.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sagms.h"
#include "internal.h"
#include "kernels.h"

using namespace sagms;
using namespace sagms_kernels;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky launch error so later calls are not poisoned
    return fail(e == cudaErrorMemoryAllocation ? SAGMS_ERR_OOM : SAGMS_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

int round_up(int x, int k) { return (x + k - 1) / k * k; }



// colQ layout of a column-indexed shape: [K][DC][T], byte offset 4 * col of check
// tg + k * T in slot qslot[e] (4 * NP, the padding column, for padding).
std::vector<uint32_t> qc_layout(int m, const int32_t* row_ptr, const int32_t* col_idx, const std::vector<int>& qslot,
                                const QcVariant& V) {
    std::vector<uint32_t> out((size_t)V.k * V.dc * V.t, (uint32_t)V.np * 4u);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            out[((size_t)(i / V.t) * V.dc + qslot[e]) * V.t + (i % V.t)] = (uint32_t)col_idx[e] * 4u;
    return out;
}

// True when slot[e] mod D differs between the edges of every qubit (the column-indexed
// kernel keeps qubit c's edge in slot j at message row j mod D of column c).
bool column_slots_ok(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, const std::vector<int>& slot,
                     int D) {
    std::vector<uint32_t> used(n, 0u);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const uint32_t bit = 1u << (slot[e] % D);
            if (used[col_idx[e]] & bit) return false;
            used[col_idx[e]] |= bit;
        }
    return true;
}

// Column-indexed slots for any code whose degrees fit the shape (dv <= D, dc <= 2D), by edge
// colouring.  Each check's edges split, in CSR order, into two halves of at most D edges; the
// bipartite graph of qubits and check halves then has maximum degree D, so by Koenig's
// edge-colouring theorem it has a proper colouring with D colours, found here by the
// alternating-path method: give an edge a colour free at both ends, or else take a colour a
// free at its qubit and b free at its half, swap a and b along the a/b path leaving the half
// (the path cannot reach the qubit, the graph being bipartite) and give the edge a.  An edge of
// colour q in half h takes slot q + D h: distinct slots within a check, distinct q at a qubit.
// Preferred colours keep shift structure where the code has it (quasi-cyclic codes listed with
// sorted columns): first the colour of the edge one check and one column back in the same
// half, then the edge's rank in its half, then any colour free at both ends.  Returns an empty vector if no colouring is found
// (it always is when the degrees fit).
std::vector<int> colour_slots(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, int D) {
    const int nnz = row_ptr[m];
    std::vector<int> colour(nnz, -1), half(nnz), rank(nnz);
    std::vector<int> at_q((size_t)n * D, -1), at_h((size_t)2 * m * D, -1);
    for (int i = 0; i < m; ++i) {
        const int d = row_ptr[i + 1] - row_ptr[i], h0 = (d + 1) / 2;
        if (h0 > D || d - h0 > D) return {};
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int r = e - row_ptr[i];
            half[e] = 2 * i + (r < h0 ? 0 : 1);
            rank[e] = r < h0 ? r : r - h0;
        }
    }
    auto free_at = [&](int e, int c) {
        return at_q[(size_t)col_idx[e] * D + c] < 0 && at_h[(size_t)half[e] * D + c] < 0;
    };
    auto set = [&](int e, int c) {
        colour[e] = c;
        at_q[(size_t)col_idx[e] * D + c] = e;
        at_h[(size_t)half[e] * D + c] = e;
    };
    std::vector<int> path;
    for (int i = 0; i < m; ++i) {
        for (int e = row_ptr[i]; i > 0 && e < row_ptr[i + 1]; ++e) {   // the shifted predecessor's colour
            for (int f = row_ptr[i - 1]; f < row_ptr[i]; ++f)
                if (col_idx[f] == col_idx[e] - 1 && (half[f] & 1) == (half[e] & 1) && colour[f] >= 0 &&
                    free_at(e, colour[f])) {
                    set(e, colour[f]);
                    break;
                }
        }
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (colour[e] >= 0) continue;
            if (free_at(e, rank[e])) { set(e, rank[e]); continue; }
            int c = 0;
            while (c < D && !free_at(e, c)) ++c;
            if (c < D) { set(e, c); continue; }
            int a = 0, b = 0;
            while (a < D && at_q[(size_t)col_idx[e] * D + a] >= 0) ++a;
            while (b < D && at_h[(size_t)half[e] * D + b] >= 0) ++b;
            if (a == D || b == D) return {};
            if (at_h[(size_t)half[e] * D + a] >= 0) {
                // alternating a/b path from the half: half -a-> qubit -b-> half -a-> ...
                path.clear();
                int x = half[e], cur = a;
                bool at_half = true;
                while ((int)path.size() <= nnz) {
                    const int f = at_half ? at_h[(size_t)x * D + cur] : at_q[(size_t)x * D + cur];
                    if (f < 0) break;
                    path.push_back(f);
                    x = at_half ? col_idx[f] : half[f];
                    at_half = !at_half;
                    cur = (cur == a) ? b : a;
                }
                for (int f : path) {
                    at_q[(size_t)col_idx[f] * D + colour[f]] = -1;
                    at_h[(size_t)half[f] * D + colour[f]] = -1;
                }
                for (int f : path) set(f, colour[f] == a ? b : a);
            }
            if (!free_at(e, a)) return {};
            set(e, a);
        }
    }
    std::vector<int> slot(nnz);
    for (int e = 0; e < nnz; ++e) slot[e] = colour[e] + D * (half[e] & 1);
    if (!column_slots_ok(m, n, row_ptr, col_idx, slot, D)) return {};
    return slot;
}

// CSR checks shared by the entry points that take a matrix: row_ptr monotone from 0 to nnz,
// columns in range, no repeated column in a row.  Reports the largest check and qubit degrees.
int check_csr(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, int* dc_max,
              int* dv_max) {
    if (!row_ptr || (nnz > 0 && !col_idx)) return fail(SAGMS_ERR_ARG, "row_ptr/col_idx is NULL");
    if (m < 1 || n < 1 || nnz < 0) return fail(SAGMS_ERR_ARG, "need m >= 1, n >= 1, nnz >= 0");
    if (row_ptr[0] != 0 || row_ptr[m] != nnz) return fail(SAGMS_ERR_CSR, "row_ptr[0] must be 0 and row_ptr[m] == nnz");
    int dc = 0;
    std::vector<int> deg_v(n, 0);
    std::vector<int> seen(n, -1);
    for (int i = 0; i < m; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return fail(SAGMS_ERR_CSR, "row_ptr not monotone at row %d", i);
        dc = std::max(dc, row_ptr[i + 1] - row_ptr[i]);
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int j = col_idx[e];
            if (j < 0 || j >= n) return fail(SAGMS_ERR_CSR, "column %d out of range in row %d", j, i);
            if (seen[j] == i) return fail(SAGMS_ERR_CSR, "duplicate column %d in row %d", j, i);
            seen[j] = i;
            deg_v[j]++;
        }
    }
    *dc_max = dc;
    *dv_max = *std::max_element(deg_v.begin(), deg_v.end());
    return SAGMS_OK;
}

// First-fit layers of the checks in index order: check i joins the smallest layer that no
// earlier check sharing a qubit with it uses, so the checks of a layer share no qubit.
// order: the checks by (layer, index); lay_ptr[l]: position of layer l's first check.
void first_fit_layers(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, std::vector<int>& order,
                      std::vector<int>& lay_ptr) {
    std::vector<int> cptr(n + 1, 0), cchk(row_ptr[m]);
    for (int e = 0; e < row_ptr[m]; ++e) cptr[col_idx[e] + 1]++;
    for (int j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    {
        std::vector<int> fill(cptr.begin(), cptr.end() - 1);
        for (int i = 0; i < m; ++i)
            for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) cchk[fill[col_idx[e]]++] = i;
    }
    std::vector<int> layer(m, 0), seen(m + 1, -1);
    int L = 0;
    for (int i = 0; i < m; ++i) {
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            for (int u = cptr[col_idx[e]]; u < cptr[col_idx[e] + 1]; ++u)
                if (cchk[u] < i) seen[layer[cchk[u]]] = i;
        int l = 0;
        while (seen[l] == i) ++l;
        layer[i] = l;
        L = std::max(L, l + 1);
    }
    lay_ptr.assign(L + 1, 0);
    for (int i = 0; i < m; ++i) lay_ptr[layer[i] + 1]++;
    for (int l = 0; l < L; ++l) lay_ptr[l + 1] += lay_ptr[l];
    order.assign(m, 0);
    std::vector<int> fill(lay_ptr.begin(), lay_ptr.end() - 1);
    for (int i = 0; i < m; ++i) order[fill[layer[i]]++] = i;
}

// Proper D-edge-colouring of a bipartite multigraph whose vertex degrees are at most D
// (Koenig's theorem), by alternating paths: an edge takes a colour a free at its left end;
// if a is taken at its right end, where b is free, the a/b path leaving the right end swaps
// its colours first.  edges[e] = (left, right).  Returns the colour of every edge.
std::vector<int> bipartite_edge_colouring(int nl, int nr, const std::vector<std::pair<int, int>>& edges, int D) {
    std::vector<int> colour(edges.size(), -1), atl((size_t)nl * D, -1), atr((size_t)nr * D, -1);
    std::vector<int> path;
    for (size_t e = 0; e < edges.size(); ++e) {
        const int u = edges[e].first, v = edges[e].second;
        int a = 0, b = 0;
        while (atl[(size_t)u * D + a] >= 0) ++a;
        while (atr[(size_t)v * D + b] >= 0) ++b;
        if (atr[(size_t)v * D + a] >= 0) {
            path.clear();
            int x = v, cur = a;
            bool right = true;
            for (;;) {
                const int f = right ? atr[(size_t)x * D + cur] : atl[(size_t)x * D + cur];
                if (f < 0) break;
                path.push_back(f);
                x = right ? edges[f].first : edges[f].second;
                right = !right;
                cur = (cur == a) ? b : a;
            }
            for (int f : path) {
                atl[(size_t)edges[f].first * D + colour[f]] = -1;
                atr[(size_t)edges[f].second * D + colour[f]] = -1;
            }
            for (int f : path) {
                colour[f] = (colour[f] == a) ? b : a;
                atl[(size_t)edges[f].first * D + colour[f]] = f;
                atr[(size_t)edges[f].second * D + colour[f]] = f;
            }
        }
        colour[e] = a;
        atl[(size_t)u * D + a] = (int)e;
        atr[(size_t)v * D + a] = (int)e;
    }
    return colour;
}

// Slot order of the records of one warp of the layered kernel (up to 32 checks that update
// together): at slot step j the warp gathers one posterior per check, and two of them in the
// same shared-memory bank (column mod 32) serialise.  Each bank is split into copies of at
// most DC columns, and the graph of checks and bank copies is DC-edge-coloured: colour j is
// the slot of a column, so at every step a bank serves at most as many columns as it has
// copies, ceil(columns in the bank / DC).  rows[k]: the columns of the warp's k-th check;
// out[k][j]: the column in slot j, pad where none.
void warp_slot_order(const std::vector<std::vector<int>>& rows, int DC, int pad, std::vector<std::vector<int>>& out) {
    std::vector<std::pair<int, int>> edges;
    std::vector<int> ecol, deg(32, 0);
    int ncopies = 0;
    std::vector<std::vector<int>> bank_copies(32);
    for (size_t k = 0; k < rows.size(); ++k)
        for (int c : rows[k]) {
            const int b = c & 31;
            const int cp = deg[b]++ / DC;
            if ((int)bank_copies[b].size() <= cp) bank_copies[b].push_back(ncopies++);
            edges.push_back({(int)k, bank_copies[b][cp]});
            ecol.push_back(c);
        }
    const std::vector<int> colour = bipartite_edge_colouring((int)rows.size(), ncopies, edges, DC);
    out.assign(rows.size(), std::vector<int>(DC, pad));
    for (size_t e = 0; e < edges.size(); ++e) out[edges[e].first][colour[e]] = ecol[e];
}

// Threads per CTA of the layered kernel for a largest layer of lay_max checks: at most two
// checks per thread in the largest layer (measured at GB(1023,5), largest layer 85: 64
// threads 3.2e7 shots/s, 128 threads 3.05e7, 32 threads 2.8e7; codes with layers of at most
// 64 checks run fastest with 32).
int layered_threads(int lay_max) { return lay_max <= 64 ? 32 : (lay_max <= 128 ? 64 : 128); }

// Column-indexed slots of a code for D message rows: the CSR order when it already gives every
// qubit distinct slots mod D, else an edge colouring (empty if neither).
std::vector<int> column_slots(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, int D) {
    std::vector<int> slot(row_ptr[m]);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) slot[e] = e - row_ptr[i];
    if (column_slots_ok(m, n, row_ptr, col_idx, slot, D)) return slot;
    return colour_slots(m, n, row_ptr, col_idx, D);
}

constexpr int kMaxDevices = 64;

// Autotune cache: when SAGMS_AUTOTUNE_CACHE names a file, sagms_autotune appends
// "<code fingerprint hex> <packed plan>" lines to it and sagms_load_code takes the last
// plan recorded for the code's fingerprint.
uint32_t cached_plan(uint64_t key) {
    const char* path = std::getenv("SAGMS_AUTOTUNE_CACHE");
    if (!path || !*path) return 0u;
    FILE* f = std::fopen(path, "r");
    if (!f) return 0u;
    unsigned long long k = 0;
    unsigned int pl = 0;
    uint32_t found = 0u;
    while (std::fscanf(f, "%llx %u", &k, &pl) == 2)
        if ((uint64_t)k == key) found = pl;
    std::fclose(f);
    return found;
}

void store_cached_plan(uint64_t key, uint32_t pl) {
    const char* path = std::getenv("SAGMS_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%016llx %u\n", (unsigned long long)key, pl);
    std::fclose(f);
}

using sagms_internal::Plan;
Plan unpack_plan(uint32_t v) {
    Plan p;
    p.kernel = (int)(v & 7u);
    p.ctas_per_sm = (int)((v >> 8) & 0xffu);
    p.chunk_lg = (int)((v >> 16) & 0xfu);
    return p;
}
uint32_t pack_plan(const Plan& p) {
    return (uint32_t)(p.kernel & 7) | ((uint32_t)(p.ctas_per_sm & 0xff) << 8) | ((uint32_t)(p.chunk_lg & 0xf) << 16);
}

// Largest launch of a continuous-batching kernel: its per-shot indexing (shot * words per pattern)
// stays within 32-bit integers.
long long max_slot_chunk(int m, int n) {
    const long long words = std::max((m + 31) / 32, (n + 31) / 32);
    return 0x7fffffffLL / std::max(1LL, words);
}

// Shots per claimed chunk of the continuous-batching kernels (log2): about eight chunks per CTA, at
// least 2 shots (the claim ring needs a chunk of slack per refill round) and at most 16.
int chunk_lg_for(long long shots, long long grid) {
    int lg = 1;
    while (lg < 4 && (shots >> (lg + 1)) >= grid * 8) ++lg;
    return lg;
}


}  // namespace

struct sagms_code {
    int m, n, nnz;
    int dc_max, dv_max;
    int variant, DC, DV;
    int Mp, Np;
    int device;
    uint16_t* d_colT;
    uint16_t* d_vneT;
    int slot_variant;      // -1: no two-slot kernel for this shape
    uint16_t* d_colB;      // [DC][MP] byte offsets into P2
    uint32_t* d_vneB;      // [DV][NP] byte offsets into C2
    bool groups;           // the two-group kernel covers this code
    uint16_t* d_colG;      // [2][kGroupDC][1024] byte offsets of P_g entries
    uint32_t* d_vneG;      // [2][kGroupDV][2048] byte offsets of C_g entries
    int qc_variant;        // -1: no column-indexed kernel for this code
    uint32_t* d_colQ;      // qc_layout
    int qc_bp_variant;     // -1: no BP column-indexed shape (kQcBpVariants) for this code
    uint32_t* d_colQbp;    // qc_layout for it
    uint16_t* d_qchk;      // [dv_max][n] checks of each qubit, 0xFFFF padding (Monte Carlo sampler)
    int lay_variant;       // -1: no layered-schedule kernel for this code (check degree above 24)
    int lay_L;             // layers of the first-fit partition
    int lay_max;           // checks in the largest layer
    uint32_t* d_lrec;      // [m][R] check records in layer order (LayeredRec)
    int* d_lptr;           // [lay_L + 1] first position of each layer
    uint16_t* d_lqe;       // [n][dv_max] edges of each qubit (layer position << 5 | slot), 0xFFFF pads
    int k_logicals;        // logical operators attached for the Monte Carlo check (-1: none)
    uint32_t* d_logicals;  // [k][ceil(n/32)]
    // Launch plan chosen by sagms_autotune (0 = defaults), packed so decodes on other
    // threads read it atomically: bits 0-2 kernel (0 auto, 1 one-shot-per-CTA, 2 two-slot,
    // 3 two-group, 4 two-group with column-indexed messages),
    // bits 8-15 CTAs per SM (0 = occupancy limit), bits 16-19 log2 shots per claimed chunk
    // (0 = automatic).
    mutable std::atomic<uint32_t> plan;
    // Largest launch of a continuous-batching kernel set by sagms_set_launch_limit (0: only the
    // 32-bit indexing bound of max_slot_chunk applies).
    std::atomic<long long> launch_limit{0};
    uint64_t shape_key;    // code fingerprint for the autotune cache
};

namespace {

// Shots per launch of a continuous-batching kernel for this code: the 32-bit indexing bound,
// lowered to the code's launch limit when one is set.
long long launch_chunk(const sagms_code* code) {
    const long long cap = max_slot_chunk(code->m, code->n);
    const long long lim = code->launch_limit.load();
    return lim > 0 ? std::min(cap, lim) : cap;
}

}  // namespace

extern "C" {

const char* sagms_last_error_string(void) { return g_last_error.c_str(); }

const char* sagms_version(void) {
    static char buf[256];
    static std::once_flag once;
    std::call_once(once, [] {
        snprintf(buf, sizeof(buf),
                 "libsagms 0.1 sm_103a; msfam_clip=%g bp_clip=%g max_dc=%d max_dv=%d max_m=%d qc_tmem=%d",
                 (double)kMsFamClip, (double)kBpClip, SAGMS_MAX_DC, SAGMS_MAX_DV, SAGMS_MAX_M,
                 sagms::QcShape<10, 5, 4, 256, 2048>::TM ? 1 : 0);
    });
    return buf;
}

double sagms_alpha_star(double L0, int32_t dc) {
    if (!(L0 > 0.0) || dc < 2) return NAN;
    return 2.0 * std::atanh(std::pow(std::tanh(0.5 * L0), (double)(dc - 1))) / L0;
}

// Smallest alpha_min accepted.  Eq. 7's gain is at least alpha_min > 0 in exact arithmetic; in
// FP32 the term (alpha_max - alpha_min) * |s~|_0 / m can round above alpha_max - alpha_min by
// about 2^-22 alpha_max, so alpha_min >= 2^-20 (alpha_max <= 1) keeps every computed gain
// positive, which the kernels' check-node arithmetic relies on.
constexpr float kMinAlphaMin = 0x1p-20f;

int sagms_check_params(const sagms_params* p) {
    if (!p) return fail(SAGMS_ERR_ARG, "params is NULL");
    if (p->flags & ~(uint32_t)(SAGMS_FLAG_L0_PER_QUBIT | SAGMS_FLAG_NO_EARLY_STOP | SAGMS_FLAG_GENERIC_KERNEL |
                               SAGMS_FLAG_AUTO_CEILING | SAGMS_FLAG_LAYERED))
        return fail(SAGMS_ERR_ARG, "unknown flag bits 0x%x", p->flags);
    if ((p->flags & SAGMS_FLAG_LAYERED) && p->mode == SAGMS_BP)
        return fail(SAGMS_ERR_PARAM, "SAGMS_FLAG_LAYERED applies to the MS family only");
    const bool auto_ceiling = (p->flags & SAGMS_FLAG_AUTO_CEILING) != 0;
    if (auto_ceiling && p->mode != SAGMS_SAGMS)
        return fail(SAGMS_ERR_PARAM, "SAGMS_FLAG_AUTO_CEILING applies to the SAGMS mode only");
    if (auto_ceiling && (p->flags & SAGMS_FLAG_L0_PER_QUBIT))
        return fail(SAGMS_ERR_PARAM, "SAGMS_FLAG_AUTO_CEILING needs one prior per shot");
    if (p->max_iter < 0 || p->max_iter > 100000)
        return fail(SAGMS_ERR_PARAM, "max_iter %d outside [0, 100000]", p->max_iter);
    switch (p->mode) {
        case SAGMS_MS:
        case SAGMS_BP:
            return SAGMS_OK;
        case SAGMS_SMS:
            if (!(p->alpha > 0.0f && p->alpha <= 1.0f))
                return fail(SAGMS_ERR_PARAM, "SMS alpha %g outside (0, 1]", (double)p->alpha);
            return SAGMS_OK;
        case SAGMS_SAGMS: {
            const float eta = (p->eta_unsat == 0.0f) ? 1.10f : p->eta_unsat;
            if (auto_ceiling) {
                // alpha_max comes from each shot's prior, clamped to [alpha_min, 1/eta]
                if (!(p->alpha_min >= kMinAlphaMin && p->alpha_min <= 1.0f))
                    return fail(SAGMS_ERR_PARAM, "need 2^-20 <= alpha_min <= 1 (got %g)", (double)p->alpha_min);
                if (!(eta >= 1.0f) || !std::isfinite(eta))
                    return fail(SAGMS_ERR_PARAM, "eta_unsat %g must be >= 1", (double)eta);
                if ((double)p->alpha_min * (double)eta > 1.0 + 1e-6)
                    return fail(SAGMS_ERR_PARAM, "stability constraint alpha_min * eta_unsat <= 1 violated (%g)",
                                (double)p->alpha_min * (double)eta);
                return SAGMS_OK;
            }
            if (!(p->alpha_min >= kMinAlphaMin && p->alpha_min <= p->alpha_max && p->alpha_max <= 1.0f))
                return fail(SAGMS_ERR_PARAM, "need 2^-20 <= alpha_min <= alpha_max <= 1 (got %g, %g)",
                            (double)p->alpha_min, (double)p->alpha_max);
            if (!(eta >= 1.0f) || !std::isfinite(eta))
                return fail(SAGMS_ERR_PARAM, "eta_unsat %g must be >= 1", (double)eta);
            if ((double)p->alpha_max * (double)eta > 1.0 + 1e-6)
                return fail(SAGMS_ERR_PARAM, "stability constraint alpha_max * eta_unsat <= 1 violated (%g)",
                            (double)p->alpha_max * (double)eta);
            return SAGMS_OK;
        }
        default:
            return fail(SAGMS_ERR_PARAM, "unknown mode %d", p->mode);
    }
}

}  // extern "C"

namespace {
__global__ void phi_kernel(const float* __restrict__ x, float* __restrict__ y, long long n, int form) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = form ? phi_ref(x[i]) : phi_fn(x[i]);
}
}  // namespace

extern "C" {

int sagms_phi(const float* d_x, float* d_y, int64_t n, int32_t form, void* stream) {
    if (n < 0 || (n > 0 && (!d_x || !d_y))) return fail(SAGMS_ERR_ARG, "bad phi arguments");
    if (form != 0 && form != 1) return fail(SAGMS_ERR_ARG, "unknown phi form %d", form);
    if (n == 0) return SAGMS_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    phi_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_x, d_y, n, form);
    const cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? SAGMS_OK : cuda_fail(ce, "phi launch");
}

int sagms_check_layers(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                       int32_t* layer, int32_t* num_layers) {
    if (!layer) return fail(SAGMS_ERR_ARG, "layer is NULL");
    int dc_max = 0, dv_max = 0;
    const int rc = check_csr(m, n, nnz, row_ptr, col_idx, &dc_max, &dv_max);
    if (rc != SAGMS_OK) return rc;
    std::vector<int> order, lay_ptr;
    first_fit_layers(m, n, row_ptr, col_idx, order, lay_ptr);
    for (size_t l = 0; l + 1 < lay_ptr.size(); ++l)
        for (int p = lay_ptr[l]; p < lay_ptr[l + 1]; ++p) layer[order[p]] = (int32_t)l;
    if (num_layers) *num_layers = (int32_t)lay_ptr.size() - 1;
    return SAGMS_OK;
}

int sagms_column_slots(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                       int32_t D, int32_t* slots) {
    if (!slots && nnz > 0) return fail(SAGMS_ERR_ARG, "slots is NULL");
    int dc_max = 0, dv_max = 0;
    const int rc = check_csr(m, n, nnz, row_ptr, col_idx, &dc_max, &dv_max);
    if (rc != SAGMS_OK) return rc;
    if (D < 1 || D > 32) return fail(SAGMS_ERR_ARG, "D = %d outside [1, 32]", D);
    if (dv_max > D || dc_max > 2 * D)
        return fail(SAGMS_ERR_DEGREE, "degrees dc=%d dv=%d need more than %d message rows", dc_max, dv_max, D);
    if (nnz == 0) return SAGMS_OK;   // no edges: the empty assignment
    const std::vector<int> s = column_slots(m, n, row_ptr, col_idx, D);
    if (s.empty()) return fail(SAGMS_ERR_DEGREE, "no column-indexed slot assignment found");
    std::copy(s.begin(), s.end(), slots);
    return SAGMS_OK;
}

int sagms_load_code(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                    sagms_code** out) {
    if (!out) return fail(SAGMS_ERR_ARG, "out is NULL");
    *out = nullptr;
    int dc_max = 0, dv_max = 0;
    const int rc = check_csr(m, n, nnz, row_ptr, col_idx, &dc_max, &dv_max);
    if (rc != SAGMS_OK) return rc;
    if (m > SAGMS_MAX_M) return fail(SAGMS_ERR_SIZE, "m = %d exceeds %d checks", m, SAGMS_MAX_M);
    if (n > 60000) return fail(SAGMS_ERR_SIZE, "n = %d too large", n);
    if (dc_max > SAGMS_MAX_DC || dv_max > SAGMS_MAX_DV)
        return fail(SAGMS_ERR_DEGREE, "degrees dc=%d dv=%d exceed limits %d/%d", dc_max, dv_max, SAGMS_MAX_DC,
                    SAGMS_MAX_DV);
    // Column-indexed shape: the first compiled one whose degrees and size class fit.
    int qv = -1;
    for (int v = 0; v < num_qc_variants() && qv < 0; ++v) {
        const QcVariant& V = qc_variant(v);
        if (dc_max > V.dc || dv_max > V.dv) continue;
        if (m > V.k * V.t || 2 * m <= V.k * V.t || n > V.np || 2 * n <= V.np) continue;
        qv = v;
    }
    // Edge order shared by every layout, so that all kernels add each qubit's messages in the
    // same order (bitwise-identical results): cslot[e] = the check slot of edge e in the
    // slot-major layouts, vrow[e] = its row in the qubit's variable-node sum.  With a
    // column-indexed shape, qslot[e] = its slot there (the CSR order when that already gives
    // every qubit distinct slots mod DV, else an edge colouring), cslot its rank in the check
    // by qslot and vrow = qslot mod DV; otherwise cslot is the CSR order and vrow the rank among
    // the qubit's edges by (cslot, check).
    std::vector<int> cslot(nnz), qslot, vrow(nnz);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) cslot[e] = e - row_ptr[i];
    int DVr = dv_max;   // message rows every variable-node layout needs
    if (qv >= 0) {
        const int DVq = qc_variant(qv).dv;
        qslot = column_slots(m, n, row_ptr, col_idx, DVq);
        if (qslot.empty()) {
            qv = -1;
        } else {
            DVr = DVq;
            for (int i = 0; i < m; ++i) {
                std::vector<std::pair<int, int>> r;
                for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) r.push_back({qslot[e], e});
                std::sort(r.begin(), r.end());
                for (size_t k = 0; k < r.size(); ++k) cslot[r[k].second] = (int)k;
            }
            for (int64_t e = 0; e < nnz; ++e) vrow[e] = qslot[e] % DVq;
        }
    }
    // vedges[c] = (vrow, check, cslot) of qubit c's edges
    std::vector<std::vector<std::array<int, 3>>> vedges(n);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) vedges[col_idx[e]].push_back({cslot[e], i, e});
    for (int c = 0; c < n; ++c) {
        auto& ve = vedges[c];
        std::sort(ve.begin(), ve.end());   // by (cslot, check): consecutive qubits of a circulant, consecutive positions
        for (size_t q = 0; q < ve.size(); ++q) {
            const int e = ve[q][2];
            ve[q] = {qv >= 0 ? vrow[e] : (int)q, ve[q][1], cslot[e]};
        }
    }

    int variant = kNumVariants - 1;
    for (int v = 0; v < kNumVariants; ++v)
        if (kVariants[v].dc >= dc_max && kVariants[v].dv >= DVr) { variant = v; break; }
    const int DC = kVariants[variant].dc, DV = kVariants[variant].dv;
    const int Mp = round_up(m, 32);
    const int Np = round_up(n + 1, 32);
    if ((long long)DC * Mp + 1 > 65535) return fail(SAGMS_ERR_SIZE, "edge slots exceed 16-bit indexing");

    // Slot-major layouts.  colT[j*Mp + i] = column of the edge of check i in slot j (n = padding).
    std::vector<uint16_t> colT((size_t)DC * Mp, (uint16_t)n);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            colT[(size_t)cslot[e] * Mp + i] = (uint16_t)col_idx[e];
    // vneT[q*Np + c] = slot position of qubit c's edge in message row q
    std::vector<uint16_t> vneT((size_t)DV * Np, (uint16_t)(DC * Mp));
    for (int c = 0; c < n; ++c)
        for (const auto& x : vedges[c]) vneT[(size_t)x[0] * Np + c] = (uint16_t)(x[2] * Mp + x[1]);

    // Two-slot layout, when a compiled shape covers the code.
    int sv = -1;
    for (int v = 0; v < kNumSlotVariants; ++v) {
        const SlotVariant& S = kSlotVariants[v];
        if (dc_max <= S.dc && DVr <= S.dv && m <= S.mp && S.mp <= 2 * round_up(m, 32) &&
            n <= S.np && S.np * 8 < 65536) { sv = v; break; }
    }
    std::vector<uint16_t> colB;
    std::vector<uint32_t> vneB;
    if (sv >= 0) {
        const SlotVariant& S = kSlotVariants[sv];
        colB.assign((size_t)S.dc * S.mp, (uint16_t)(S.np * 8));   // padding -> sentinel qubit NP
        for (int i = 0; i < m; ++i)
            for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                colB[(size_t)cslot[e] * S.mp + i] = (uint16_t)(col_idx[e] * 8);
        vneB.assign((size_t)S.dv * S.np, (uint32_t)(S.dc * S.mp * 8));
        for (int c = 0; c < n; ++c)
            for (const auto& x : vedges[c]) vneB[(size_t)x[0] * S.np + c] = (uint32_t)((x[2] * S.mp + x[1]) * 8);
    }

    // Two-group layout: the same graph once per group, as byte offsets from the start of
    // shared memory into that group's posterior and message arrays.
    const bool groups = dc_max <= kGroupDC && DVr <= kGroupDV && m > 512 && m <= kGrpChecks && n <= kGrpQubits;
    std::vector<uint16_t> colG;
    std::vector<uint32_t> vneG;
    if (groups) {
        colG.resize((size_t)2 * kGroupDC * kGrpChecks);
        vneG.resize((size_t)2 * kGroupDV * kGrpQubits);
        for (int g = 0; g < 2; ++g) {
            uint16_t* cg = colG.data() + (size_t)g * kGroupDC * kGrpChecks;
            uint32_t* vg = vneG.data() + (size_t)g * kGroupDV * kGrpQubits;
            const size_t pb = grp_P_off(g), cb = grp_C_off(kGroupDC, g);
            std::fill(cg, cg + kGroupDC * kGrpChecks, (uint16_t)(pb + (size_t)kGrpQubits * 4));
            for (int i = 0; i < m; ++i)
                for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                    cg[(size_t)cslot[e] * kGrpChecks + i] = (uint16_t)(pb + (size_t)col_idx[e] * 4);
            std::fill(vg, vg + kGroupDV * kGrpQubits, (uint32_t)(cb + (size_t)kGroupDC * kGrpChecks * 4));
            for (int c = 0; c < n; ++c)
                for (const auto& x : vedges[c])
                    vg[(size_t)x[0] * kGrpQubits + c] = (uint32_t)(cb + ((size_t)x[2] * kGrpChecks + x[1]) * 4);
        }
    }

    std::vector<uint32_t> colQ;
    if (qv >= 0) colQ = qc_layout(m, row_ptr, col_idx, qslot, qc_variant(qv));
    // BP's column-indexed shape: the same message rows (so the same slots), filled at least
    // halfway, as for the shape above.
    int bpv = -1;
    std::vector<uint32_t> colQbp;
    for (int v = 0; qv >= 0 && v < kNumQcBp && bpv < 0; ++v) {
        const QcVariant& V = kQcBpVariants[v];
        if (V.dv != qc_variant(qv).dv || dc_max > V.dc) continue;
        if (m > V.k * V.t || 2 * m <= V.k * V.t || n > V.np || 2 * n <= V.np) continue;
        bpv = v;
    }
    if (bpv >= 0) colQbp = qc_layout(m, row_ptr, col_idx, qslot, kQcBpVariants[bpv]);

    // Layered schedule: first-fit layers and, in layer order, each check's record (columns,
    // padding n, then the check index and its degree).
    int lv = -1, lay_max = 0;
    std::vector<int> lorder, lptr;
    std::vector<uint32_t> lrec;
    std::vector<uint16_t> lqe;
    first_fit_layers(m, n, row_ptr, col_idx, lorder, lptr);
    for (size_t l = 0; l + 1 < lptr.size(); ++l) lay_max = std::max(lay_max, lptr[l + 1] - lptr[l]);
    for (int v = 0; v < kNumLayeredVariants && lv < 0; ++v) {
        const LayeredVariant& V = kLayeredVariants[v];
        if (dc_max <= V.dc && V.t == layered_threads(lay_max)) lv = v;
    }
    if (lv >= 0) {
        // the kernel's warps take 32 consecutive positions from the start of each layer; their
        // slot orders spread each step's posterior gathers over the shared-memory banks
        const int DCl = kLayeredVariants[lv].dc, R = (DCl + 1 + 3) / 4 * 4;   // LayeredRec<DCl>::R
        lrec.assign((size_t)m * R, 0u);
        std::vector<std::vector<int>> rows, slots;
        for (size_t l = 0; l + 1 < lptr.size(); ++l)
            for (int w0 = lptr[l]; w0 < lptr[l + 1]; w0 += 32) {
                const int w1 = std::min(w0 + 32, lptr[l + 1]);
                rows.assign(w1 - w0, {});
                for (int p = w0; p < w1; ++p)
                    for (int e = row_ptr[lorder[p]]; e < row_ptr[lorder[p] + 1]; ++e) rows[p - w0].push_back(col_idx[e]);
                warp_slot_order(rows, DCl, n, slots);
                for (int p = w0; p < w1; ++p) {
                    uint32_t* r = lrec.data() + (size_t)p * R;
                    for (int j = 0; j < DCl; ++j) r[j] = 4u * (uint32_t)slots[p - w0][j];
                    r[DCl] = (uint32_t)lorder[p] | ((uint32_t)(row_ptr[lorder[p] + 1] - row_ptr[lorder[p]]) << 16);
                }
            }
        // qubit-to-edge lists for the posterior rebuild, in layer-position order
        lqe.assign((size_t)n * std::max(dv_max, 1), (uint16_t)0xFFFFu);
        std::vector<int> fillq(n, 0);
        for (int p = 0; p < m; ++p)
            for (int j = 0; j < DCl; ++j) {
                const uint32_t o = lrec[(size_t)p * R + j];
                if (o == 4u * (uint32_t)n) continue;
                const int c = (int)(o / 4u);
                lqe[(size_t)c * dv_max + fillq[c]++] = (uint16_t)((p << 5) | j);
            }
    }

    // Checks of each qubit, for syndrome formation in the Monte Carlo sampler.
    std::vector<uint16_t> qchk((size_t)dv_max * n, (uint16_t)0xFFFFu);
    for (int c = 0; c < n; ++c)
        for (size_t q = 0; q < vedges[c].size(); ++q) qchk[q * n + c] = (uint16_t)vedges[c][q][1];

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    sagms_code* code = new sagms_code();
    code->qc_variant = qv;
    code->lay_variant = lv;
    code->lay_L = (int)lptr.size() - 1;
    code->lay_max = lay_max;
    code->d_lrec = nullptr;
    code->d_lptr = nullptr;
    code->d_lqe = nullptr;
    code->d_qchk = nullptr;
    code->k_logicals = -1;
    code->d_logicals = nullptr;
    code->d_colQ = nullptr;
    code->qc_bp_variant = bpv;
    code->d_colQbp = nullptr;
    code->slot_variant = sv;
    code->d_colB = nullptr;
    code->d_vneB = nullptr;
    code->groups = groups;
    code->d_colG = nullptr;
    code->d_vneG = nullptr;
    code->plan.store(0u);
    {
        uint64_t h = 1469598103934665603ull;   // FNV-1a over the CSR
        auto mix = [&](uint64_t x) { h = (h ^ x) * 1099511628211ull; };
        mix((uint64_t)m); mix((uint64_t)n); mix((uint64_t)nnz);
        for (int i = 0; i <= m; ++i) mix((uint64_t)(uint32_t)row_ptr[i]);
        for (int64_t e = 0; e < nnz; ++e) mix((uint64_t)(uint32_t)col_idx[e]);
        code->shape_key = h;
    }
    code->plan.store(cached_plan(code->shape_key));
    code->m = m; code->n = n; code->nnz = (int)nnz;
    code->dc_max = dc_max; code->dv_max = dv_max;
    code->variant = variant; code->DC = DC; code->DV = DV;
    code->Mp = Mp; code->Np = Np; code->device = dev;
    code->d_colT = nullptr; code->d_vneT = nullptr;
    ce = cudaMalloc(&code->d_colT, colT.size() * sizeof(uint16_t));
    if (ce == cudaSuccess) ce = cudaMalloc(&code->d_vneT, vneT.size() * sizeof(uint16_t));
    if (ce == cudaSuccess) ce = cudaMemcpy(code->d_colT, colT.data(), colT.size() * 2, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(code->d_vneT, vneT.data(), vneT.size() * 2, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && sv >= 0) {
        ce = cudaMalloc(&code->d_colB, colB.size() * sizeof(uint16_t));
        if (ce == cudaSuccess) ce = cudaMalloc(&code->d_vneB, vneB.size() * sizeof(uint32_t));
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_colB, colB.data(), colB.size() * 2, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_vneB, vneB.data(), vneB.size() * 4, cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess && groups) {
        ce = cudaMalloc(&code->d_colG, colG.size() * sizeof(uint16_t));
        if (ce == cudaSuccess) ce = cudaMalloc(&code->d_vneG, vneG.size() * sizeof(uint32_t));
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_colG, colG.data(), colG.size() * 2, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_vneG, vneG.data(), vneG.size() * 4, cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess && qv >= 0) {
        ce = cudaMalloc(&code->d_colQ, colQ.size() * sizeof(uint32_t));
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_colQ, colQ.data(), colQ.size() * 4, cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess && bpv >= 0) {
        ce = cudaMalloc(&code->d_colQbp, colQbp.size() * sizeof(uint32_t));
        if (ce == cudaSuccess)
            ce = cudaMemcpy(code->d_colQbp, colQbp.data(), colQbp.size() * 4, cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess && lv >= 0) {
        ce = cudaMalloc(&code->d_lrec, lrec.size() * sizeof(uint32_t));
        if (ce == cudaSuccess) ce = cudaMalloc(&code->d_lptr, lptr.size() * sizeof(int));
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_lrec, lrec.data(), lrec.size() * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_lptr, lptr.data(), lptr.size() * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMalloc(&code->d_lqe, lqe.size() * sizeof(uint16_t));
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_lqe, lqe.data(), lqe.size() * 2, cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess) {
        ce = cudaMalloc(&code->d_qchk, qchk.size() * sizeof(uint16_t));
        if (ce == cudaSuccess) ce = cudaMemcpy(code->d_qchk, qchk.data(), qchk.size() * 2, cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) {
        cudaFree(code->d_qchk);
        cudaFree(code->d_colT);
        cudaFree(code->d_vneT);
        cudaFree(code->d_colB);
        cudaFree(code->d_vneB);
        cudaFree(code->d_colG);
        cudaFree(code->d_vneG);
        cudaFree(code->d_colQ);
        cudaFree(code->d_colQbp);
        cudaFree(code->d_lrec);
        cudaFree(code->d_lptr);
        cudaFree(code->d_lqe);
        delete code;
        return cuda_fail(ce, "sagms_load_code upload");
    }
    *out = code;
    return SAGMS_OK;
}

void sagms_free_code(sagms_code* code) {
    if (!code) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != code->device) cudaSetDevice(code->device);
    cudaFree(code->d_colT);
    cudaFree(code->d_vneT);
    cudaFree(code->d_colB);
    cudaFree(code->d_vneB);
    cudaFree(code->d_colG);
    cudaFree(code->d_vneG);
    cudaFree(code->d_colQ);
    cudaFree(code->d_colQbp);
    cudaFree(code->d_lrec);
    cudaFree(code->d_lptr);
    cudaFree(code->d_lqe);
    cudaFree(code->d_qchk);
    cudaFree(code->d_logicals);
    if (prev >= 0 && prev != code->device) cudaSetDevice(prev);
    delete code;
}

int sagms_code_info(const sagms_code* code, int32_t* m, int32_t* n, int32_t* dc_max, int32_t* dv_max) {
    if (!code) return fail(SAGMS_ERR_ARG, "code is NULL");
    if (m) *m = code->m;
    if (n) *n = code->n;
    if (dc_max) *dc_max = code->dc_max;
    if (dv_max) *dv_max = code->dv_max;
    return SAGMS_OK;
}

int sagms_code_kernels(const sagms_code* code, uint32_t* mask) {
    if (!code || !mask) return fail(SAGMS_ERR_ARG, "code or mask is NULL");
    *mask = (1u << 1) | (code->slot_variant >= 0 ? 1u << 2 : 0u) | (code->groups ? 1u << 3 : 0u) |
            (code->qc_variant >= 0 ? 1u << 4 : 0u) | (code->qc_bp_variant >= 0 ? 1u << 5 : 0u);
    return SAGMS_OK;
}

}  // extern "C"

namespace {

// The layered-schedule kernel: one shot per CTA at a time, CTAs striding over the batch.
int launch_layered(const sagms_code* code, const DecodeArgs& a, bool per_qubit, cudaStream_t stream) {
    if (code->lay_variant < 0)
        return fail(SAGMS_ERR_DEGREE, "the layered schedule supports check degrees up to 24 (code has %d)",
                    code->dc_max);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    if (dev != code->device) return fail(SAGMS_ERR_ARG, "code was loaded on device %d, current is %d", code->device, dev);
    const LayeredVariant& V = kLayeredVariants[code->lay_variant];
    const size_t smem = layered_smem_bytes(code->Mp, code->Np, per_qubit);
    int smem_optin = 0, sms = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > (size_t)smem_optin)
        return fail(SAGMS_ERR_SIZE, "code needs %zu B of shared memory per CTA (limit %d)", smem, smem_optin);
    const void* fn = reinterpret_cast<const void*>(V.fn);
    ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaFuncSetAttribute");
    int per_sm = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, V.t, smem);
    if (ce != cudaSuccess) return cuda_fail(ce, "occupancy query");
    if (per_sm < 1) return fail(SAGMS_ERR_SIZE, "kernel does not fit on an SM");
    const long long grid = std::min<long long>(a.shots, (long long)per_sm * sms);
    const LayeredLayout lay{code->d_lrec, code->d_lptr, code->lay_L, code->d_lqe, std::max(code->dv_max, 1)};
    V.fn<<<(unsigned)grid, V.t, smem, stream>>>(a, lay);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "decode launch");
    return SAGMS_OK;
}

bool aligned4(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 3u) == 0; }

int launch_decode(const sagms_code* code, const sagms_params* p, int64_t shots, const uint32_t* d_syn,
                  const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, float* d_trace,
                  cudaStream_t stream, const Plan* plan_override = nullptr) {
    const sagms_internal::NvtxRange nvtx("sagms_decode");
    if (shots < 0) return fail(SAGMS_ERR_ARG, "shots < 0");
    if (shots > 0) {
        if (!d_syn || !d_L0 || !d_err || !d_conv || !d_iters) return fail(SAGMS_ERR_ARG, "NULL device buffer");
        // the kernels move syndrome words, priors, error words, counts and traces as 4-byte
        // elements (cp.async and plain loads/stores): a misaligned buffer would fault them
        if (!aligned4(d_syn) || !aligned4(d_L0) || !aligned4(d_err) || !aligned4(d_iters) ||
            (d_trace && !aligned4(d_trace)))
            return fail(SAGMS_ERR_ARG, "device buffers must be 4-byte aligned (uint32 / float / int32 elements)");
    }
    if (!code) return fail(SAGMS_ERR_ARG, "code is NULL");
    int rc = sagms_check_params(p);
    if (rc != SAGMS_OK) return rc;
    if (shots == 0) return SAGMS_OK;
    const bool bp = p->mode == SAGMS_BP;
    const bool per_qubit = (p->flags & SAGMS_FLAG_L0_PER_QUBIT) != 0;
    DecodeArgs a;
    a.colT = code->d_colT;
    a.vneT = code->d_vneT;
    a.m = code->m; a.n = code->n; a.Mp = code->Mp; a.Np = code->Np;
    a.mode = p->mode;
    a.alpha = p->alpha;
    a.amin = p->alpha_min;
    a.amax = p->alpha_max;
    a.eta = (p->eta_unsat == 0.0f) ? 1.10f : p->eta_unsat;
    a.inv_m = 1.0f / (float)code->m;
    a.dcmax = code->dc_max;
    a.max_iter = p->max_iter;
    a.flags = p->flags;
    a.shots = shots;
    a.syn = d_syn; a.L0 = d_L0; a.err = d_err; a.conv = d_conv; a.iters = d_iters; a.trace = d_trace;
    a.work = nullptr;
    a.chunk_lg = 1;
    if (p->flags & SAGMS_FLAG_LAYERED) return launch_layered(code, a, per_qubit, stream);

    const Plan plan = plan_override ? *plan_override : unpack_plan(code->plan.load());
    // Kernel: the plan's choice where the code and parameters allow it, else the fastest
    // that does (two-group, two-slot, one-shot-per-CTA).
    const bool msfam_fast = !bp && !(p->flags & SAGMS_FLAG_GENERIC_KERNEL);
    const bool bp_fast = bp && !per_qubit && !(p->flags & SAGMS_FLAG_GENERIC_KERNEL);   // BP: per-shot priors
    const bool auto_ceiling = (p->flags & SAGMS_FLAG_AUTO_CEILING) != 0;
    // BP on the column-indexed kernel: on its own shape (two checks per thread, two CTAs per
    // SM) where the code has one (129 to 512 and 1025 to 2048 qubits), else on the code's
    // shape up to 128 qubits.  On the larger shapes of four checks per thread (one 512-thread CTA of
    // 128-register threads per SM) BP's transcendental chains leave too few warps to hide them,
    // and the 1024-thread one-shot-per-CTA kernel is faster (plan kernel 4 still selects it).
    const bool qc_bp = bp_fast && code->qc_bp_variant >= 0 && (plan.kernel == 0 || plan.kernel == 4);
    const bool use_qc = qc_bp || ((msfam_fast || bp_fast) && code->qc_variant >= 0 &&
                                  (plan.kernel == 4 || (plan.kernel == 0 && (!bp || qc_variant(code->qc_variant).np <= 128))));
    const QcVariant* QV = qc_bp ? &kQcBpVariants[code->qc_bp_variant]
                                : (code->qc_variant >= 0 ? &qc_variant(code->qc_variant) : nullptr);
    const uint32_t* d_colQ = qc_bp ? code->d_colQbp : code->d_colQ;
    const int qc_form = bp ? 3 : (per_qubit ? 2 : (auto_ceiling ? 1 : 0));   // which instantiation
    const bool use_groups = !use_qc && msfam_fast && code->groups && !per_qubit &&
                            (plan.kernel == 0 || plan.kernel >= 3);
    const bool use_slots = !use_qc && !use_groups && msfam_fast && code->slot_variant >= 0 && plan.kernel != 1;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    if (dev != code->device) return fail(SAGMS_ERR_ARG, "code was loaded on device %d, current is %d", code->device, dev);
    int smem_optin = 0, sms = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* fn;
    size_t smem;
    int threads;
    int shots_per_cta;   // shots one CTA decodes at a time
    if (use_qc) {
        const QcVariant& V = *QV;
        fn = reinterpret_cast<const void*>(V.fn[qc_form]);
        smem = V.smem[qc_form];
        threads = kQcThreads;
        shots_per_cta = kQcThreads / V.t;   // one shot in flight per group
    } else if (use_groups) {
        fn = reinterpret_cast<const void*>(group_kernel_fn());
        smem = grp_smem_bytes(kGroupDC, kGroupDV);
        threads = 2 * kGrpThreads;
        shots_per_cta = 2;   // two shots in flight per CTA
    } else if (use_slots) {
        const SlotVariant& S = kSlotVariants[code->slot_variant];
        fn = reinterpret_cast<const void*>(kSlotVariants[code->slot_variant].fn);
        smem = slot_smem_bytes(S.dc, S.dv, S.mp, S.np, per_qubit);
        threads = S.mp;
        shots_per_cta = 2;
    } else {
        fn = reinterpret_cast<const void*>(generic_kernel(code->variant, bp));
        smem = smem_bytes(code->DC, code->DV, code->Mp, code->Np, per_qubit);
        threads = code->Mp;
        shots_per_cta = 1;
    }
    if (smem > (size_t)smem_optin)
        return fail(SAGMS_ERR_SIZE, "code needs %zu B of shared memory per CTA (limit %d)", smem, smem_optin);
    ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaFuncSetAttribute");
    int per_sm = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (ce != cudaSuccess) return cuda_fail(ce, "occupancy query");
    if (per_sm < 1) return fail(SAGMS_ERR_SIZE, "kernel does not fit on an SM");
    if (plan.ctas_per_sm > 0) per_sm = std::min(per_sm, plan.ctas_per_sm);
    const long long units = (shots + shots_per_cta - 1) / shots_per_cta;
    long long grid = std::min<long long>(units, (long long)per_sm * sms);
    if (plan.max_grid > 0) grid = std::min(grid, plan.max_grid);
    if (!use_qc && !use_groups && !use_slots) {
        generic_kernel(code->variant, bp)<<<(unsigned)grid, threads, smem, stream>>>(a);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "decode launch");
        return SAGMS_OK;
    }
    // Continuous-batching kernels: 32-bit shot indexing inside the kernel, so batches are
    // split into launches of at most max_slot_chunk shots.  Each launch gets a zeroed shot
    // counter that its CTAs claim chunks of shots from: the plan's scratch when it has one,
    // else scratch from the stream-ordered pool.
    const long long kMaxChunk = launch_chunk(code);
    const long long nchunks = (shots + kMaxChunk - 1) / kMaxChunk;
    int* d_work = plan.work;
    const bool own_work = d_work == nullptr;
    if (own_work) {
        ce = cudaMallocAsync(reinterpret_cast<void**>(&d_work), (size_t)nchunks * sizeof(int), stream);
        if (ce != cudaSuccess) return cuda_fail(ce, "work counter allocation");
    }
    ce = cudaMemsetAsync(d_work, 0, (size_t)nchunks * sizeof(int), stream);
    if (ce != cudaSuccess) {
        if (own_work) cudaFreeAsync(d_work, stream);
        return cuda_fail(ce, "work counter reset");
    }
    const SlotLayout slay{code->d_colB, code->d_vneB};
    const GroupLayout glay{code->d_colG, code->d_vneG};
    for (long long s0 = 0, ci = 0; s0 < shots; s0 += kMaxChunk, ++ci) {
        DecodeArgs c = a;
        const long long cnt = std::min(kMaxChunk, shots - s0);
        const int mw = (code->m + 31) / 32, nw = (code->n + 31) / 32;
        c.shots = cnt;
        c.syn = a.syn + s0 * mw;
        c.L0 = per_qubit ? a.L0 : a.L0 + s0;
        c.err = a.err + s0 * nw;
        c.conv = a.conv + s0;
        c.iters = a.iters + s0;
        c.trace = a.trace ? a.trace + s0 * (long long)(a.max_iter + 1) * code->n : nullptr;
        c.work = d_work + ci;
        const long long g = std::min(grid, (cnt + shots_per_cta - 1) / shots_per_cta);
        c.chunk_lg = plan.chunk_lg > 0 ? plan.chunk_lg : chunk_lg_for(cnt, g);
        if (use_qc)
            QV->fn[qc_form]<<<(unsigned)g, threads, smem, stream>>>(c, d_colQ);
        else if (use_groups)
            group_kernel_fn()<<<(unsigned)g, threads, smem, stream>>>(c, glay);
        else
            kSlotVariants[code->slot_variant].fn<<<(unsigned)g, threads, smem, stream>>>(c, slay);
    }
    ce = cudaGetLastError();
    if (own_work) cudaFreeAsync(d_work, stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "decode launch");
    return SAGMS_OK;
}

}  // namespace

namespace sagms_internal {

std::vector<int> column_slot_assignment(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, int D) {
    return column_slots(m, n, row_ptr, col_idx, D);
}

CodeView code_view(const sagms_code* code) {
    return CodeView{code->m, code->n, code->dv_max, code->device, code->d_qchk, code->k_logicals, code->d_logicals};
}

int attach_logicals(sagms_code* code, int k, const uint32_t* h_logicals) {
    const size_t words = (size_t)k * ((code->n + 31) / 32);
    uint32_t* d = nullptr;
    if (words > 0) {
        cudaError_t ce = cudaMalloc(&d, words * 4);
        if (ce == cudaSuccess) ce = cudaMemcpy(d, h_logicals, words * 4, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(ce, "logical operators upload");
        }
    }
    cudaFree(code->d_logicals);
    code->d_logicals = d;
    code->k_logicals = k;
    return SAGMS_OK;
}

int launch(const sagms_code* code, const sagms_params* params, int64_t shots, const uint32_t* d_syn,
           const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, cudaStream_t stream,
           const Plan* plan) {
    return launch_decode(code, params, shots, d_syn, d_L0, d_err, d_conv, d_iters, nullptr, stream, plan);
}

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
int cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

}  // namespace sagms_internal

extern "C" {

int sagms_decode(const sagms_code* code, const sagms_params* params, int64_t shots, const uint32_t* d_syn,
                 const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, void* stream) {
    return launch_decode(code, params, shots, d_syn, d_L0, d_err, d_conv, d_iters, nullptr,
                         static_cast<cudaStream_t>(stream));
}

int sagms_decode_trace(const sagms_code* code, const sagms_params* params, int64_t shots, const uint32_t* d_syn,
                       const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, float* d_trace,
                       void* stream) {
    if (shots > 0 && !d_trace) return fail(SAGMS_ERR_ARG, "d_trace is NULL");
    return launch_decode(code, params, shots, d_syn, d_L0, d_err, d_conv, d_iters, d_trace,
                         static_cast<cudaStream_t>(stream));
}

int sagms_decode_host(const sagms_code* code, const sagms_params* params, int64_t shots, const uint32_t* h_syn,
                      const float* h_L0, uint32_t* h_err, uint8_t* h_conv, int32_t* h_iters) {
    const sagms_internal::NvtxRange nvtx("sagms_decode_host");
    if (!code) return fail(SAGMS_ERR_ARG, "code is NULL");
    int rc = sagms_check_params(params);
    if (rc != SAGMS_OK) return rc;
    if (shots < 0) return fail(SAGMS_ERR_ARG, "shots < 0");
    if (shots == 0) return SAGMS_OK;
    if (!h_syn || !h_L0 || !h_err || !h_conv || !h_iters) return fail(SAGMS_ERR_ARG, "NULL host buffer");
    const bool per_qubit = (params->flags & SAGMS_FLAG_L0_PER_QUBIT) != 0;
    const int mw = (code->m + 31) / 32, nw = (code->n + 31) / 32;
    const int kStreams = 2;
    const int64_t chunk = std::max<int64_t>(std::min<int64_t>((shots + 7) / 8, 1 << 20), 1);
    cudaStream_t st[kStreams] = {nullptr, nullptr};
    struct Bufs { uint32_t* syn; float* L0; uint32_t* err; uint8_t* conv; int32_t* iters; } b[kStreams];
    memset(b, 0, sizeof(b));
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < kStreams && ce == cudaSuccess; ++k) ce = cudaStreamCreateWithFlags(&st[k], cudaStreamNonBlocking);
    const size_t l0_elems = per_qubit ? (size_t)code->n : (size_t)chunk;
    for (int k = 0; k < kStreams && ce == cudaSuccess; ++k) {
        ce = cudaMallocAsync((void**)&b[k].syn, (size_t)chunk * mw * 4, st[k]);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&b[k].L0, l0_elems * 4, st[k]);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&b[k].err, (size_t)chunk * nw * 4, st[k]);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&b[k].conv, (size_t)chunk, st[k]);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&b[k].iters, (size_t)chunk * 4, st[k]);
        if (ce == cudaSuccess && per_qubit)
            ce = cudaMemcpyAsync(b[k].L0, h_L0, (size_t)code->n * 4, cudaMemcpyHostToDevice, st[k]);
    }
    rc = (ce == cudaSuccess) ? SAGMS_OK : cuda_fail(ce, "sagms_decode_host setup");
    int64_t chunk_id = 0;
    for (int64_t s0 = 0; s0 < shots && rc == SAGMS_OK; s0 += chunk, ++chunk_id) {
        const int k = (int)(chunk_id % kStreams);
        const int64_t cnt = std::min(chunk, shots - s0);
        ce = cudaMemcpyAsync(b[k].syn, h_syn + s0 * mw, (size_t)cnt * mw * 4, cudaMemcpyHostToDevice, st[k]);
        if (ce == cudaSuccess && !per_qubit)
            ce = cudaMemcpyAsync(b[k].L0, h_L0 + s0, (size_t)cnt * 4, cudaMemcpyHostToDevice, st[k]);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "H2D copy"); break; }
        rc = launch_decode(code, params, cnt, b[k].syn, b[k].L0, b[k].err, b[k].conv, b[k].iters, nullptr, st[k]);
        if (rc != SAGMS_OK) break;
        ce = cudaMemcpyAsync(h_err + s0 * nw, b[k].err, (size_t)cnt * nw * 4, cudaMemcpyDeviceToHost, st[k]);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_conv + s0, b[k].conv, (size_t)cnt, cudaMemcpyDeviceToHost, st[k]);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_iters + s0, b[k].iters, (size_t)cnt * 4, cudaMemcpyDeviceToHost, st[k]);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "D2H copy"); break; }
    }
    for (int k = 0; k < kStreams; ++k) {
        if (!st[k]) continue;
        void* ptrs[5] = {b[k].syn, b[k].L0, b[k].err, b[k].conv, b[k].iters};
        for (void* ptr : ptrs)
            if (ptr) cudaFreeAsync(ptr, st[k]);
        ce = cudaStreamSynchronize(st[k]);
        if (ce != cudaSuccess && rc == SAGMS_OK) rc = cuda_fail(ce, "sagms_decode_host sync");
        cudaStreamDestroy(st[k]);
    }
    return rc;
}

// ---------------------------------------------------------------------------------------
// Allocation-free decoding.
//
// Some callers cannot allocate device memory while they decode: latency-critical serving
// threads (cudaMalloc and pool growth of cudaMallocAsync can synchronise or stall the
// device), processes that run under a fixed device-memory budget reserved at start-up, and
// host frameworks that own every allocation themselves.  sagms_decode_noalloc takes its
// only scratch -- the per-launch chunk counters the continuous-batching kernels claim shots
// from -- from
// this file-scope array instead of allocating it.  Every GPU that loads the library holds
// the array until the process exits.  All calls share it and it keeps the last call's
// contents; each call zeroes the counters it uses on its stream before launching, so calls
// that overlap on the GPU (different streams, or different host threads) race on it.
constexpr int kNoAllocCounters = SAGMS_NOALLOC_COUNTERS;
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocCounters];

namespace {

std::mutex g_noalloc_mutex;
int* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device `dev`.  In host code the array's
// name is only a host-side stand-in, so its device address must come from the runtime; that
// lookup happens once per device, with that device current, at the device's first call.
int noalloc_scratch(int dev, int** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(SAGMS_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        int* ptr = nullptr;
        const cudaError_t ce = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_scratch);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return SAGMS_OK;
}

}  // namespace

int sagms_decode_noalloc(const sagms_code* code, const sagms_params* p, int64_t shots, const uint32_t* d_syn,
                         const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, void* stream_v) {
    if (!code) return fail(SAGMS_ERR_ARG, "code is NULL");
    int rc = sagms_check_params(p);
    if (rc != SAGMS_OK) return rc;
    if (shots < 0) return fail(SAGMS_ERR_ARG, "shots < 0");
    if (shots == 0) return SAGMS_OK;
    if (!d_syn || !d_L0 || !d_err || !d_conv || !d_iters) return fail(SAGMS_ERR_ARG, "NULL device buffer");
    const long long kMaxChunk = launch_chunk(code);
    if (shots > kMaxChunk * kNoAllocCounters)
        return fail(SAGMS_ERR_SIZE, "sagms_decode_noalloc: %lld shots exceed the fixed scratch (%d counters of %lld shots)",
                    (long long)shots, kNoAllocCounters, kMaxChunk);
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    if (dev != code->device) return fail(SAGMS_ERR_ARG, "code was loaded on device %d, current is %d", code->device, dev);
    // The code's launch plan with the fixed scratch as its shot counters: the launcher then
    // only zeroes them (the one-shot-per-CTA kernel uses none).
    Plan pl = unpack_plan(code->plan.load());
    rc = noalloc_scratch(dev, &pl.work);
    if (rc != SAGMS_OK) return rc;
    return launch_decode(code, p, shots, d_syn, d_L0, d_err, d_conv, d_iters, nullptr, stream, &pl);
}

// ---------------------------------------------------------------------------------------
// Launch-plan autotuning, multi-code launches and CUDA graphs.

int sagms_autotune(const sagms_code* code, const sagms_params* params, int64_t shots, const uint32_t* d_syn,
                   const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, int32_t* out_plan,
                   float* out_shots_per_s, void* stream_v) {
    if (!code) return fail(SAGMS_ERR_ARG, "code is NULL");
    int rc = sagms_check_params(params);
    if (rc != SAGMS_OK) return rc;
    if (shots <= 0) return fail(SAGMS_ERR_ARG, "autotune needs a sample of at least one shot");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    int dev = 0, sms = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<Plan> cands;
    const bool slots_ok = params->mode != SAGMS_BP && code->slot_variant >= 0;
    const bool groups_ok = params->mode != SAGMS_BP && code->groups && !(params->flags & SAGMS_FLAG_L0_PER_QUBIT);
    const bool qc_ok = code->qc_variant >= 0 &&
                       !(params->mode == SAGMS_BP && (params->flags & SAGMS_FLAG_L0_PER_QUBIT));
    for (int kernel : {4, 3, 2, 1}) {
        if (kernel == 2 && !slots_ok) continue;
        if (kernel == 3 && !groups_ok) continue;
        if (kernel == 4 && !qc_ok) continue;
        for (int cps : {0, 2, 1}) {
            if (kernel >= 3 && cps != 0) continue;   // one 1024-thread CTA per SM
            if (kernel >= 2) {
                for (int clg : {0, 1, 2, 4}) {
                    Plan pl;
                    pl.kernel = kernel; pl.ctas_per_sm = cps; pl.chunk_lg = clg;
                    cands.push_back(pl);
                }
            } else {
                Plan pl;
                pl.kernel = kernel; pl.ctas_per_sm = cps;
                cands.push_back(pl);
            }
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    float best_ms = 0.0f;
    Plan best;
    bool have = false;
    for (const Plan& pl : cands) {
        rc = launch_decode(code, params, shots, d_syn, d_L0, d_err, d_conv, d_iters, nullptr, stream, &pl);  // warm-up
        if (rc != SAGMS_OK) continue;
        cudaEventRecord(e0, stream);
        for (int r = 0; r < 3 && rc == SAGMS_OK; ++r)
            rc = launch_decode(code, params, shots, d_syn, d_L0, d_err, d_conv, d_iters, nullptr, stream, &pl);
        cudaEventRecord(e1, stream);
        ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_fail(ce, "autotune sync"); }
        if (rc != SAGMS_OK) continue;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!have || ms < best_ms) { best_ms = ms; best = pl; have = true; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!have) return fail(SAGMS_ERR_CUDA, "autotune: no candidate plan launched");
    const uint32_t packed = pack_plan(best);
    code->plan.store(packed);
    store_cached_plan(code->shape_key, packed);
    if (out_plan) *out_plan = (int32_t)packed;
    if (out_shots_per_s) *out_shots_per_s = (float)(3.0 * (double)shots / (best_ms * 1e-3));
    return SAGMS_OK;
}

int sagms_set_launch_limit(sagms_code* code, int64_t shots) {
    if (!code) return fail(SAGMS_ERR_ARG, "code is NULL");
    if (shots < 0) return fail(SAGMS_ERR_ARG, "launch limit %lld < 0", (long long)shots);
    code->launch_limit.store((long long)shots);
    return SAGMS_OK;
}

int sagms_set_plan(sagms_code* code, int32_t plan) {
    if (!code) return fail(SAGMS_ERR_ARG, "code is NULL");
    if (((uint32_t)plan & ~0xfff07u) || ((uint32_t)plan & 7u) > 4u)
        return fail(SAGMS_ERR_ARG, "unknown bits in plan 0x%x", (unsigned)plan);
    code->plan.store((uint32_t)plan);
    return SAGMS_OK;
}

int sagms_decode_multi(const sagms_job* jobs, int32_t njobs, void* stream_v) {
    if (njobs < 0 || (njobs > 0 && !jobs)) return fail(SAGMS_ERR_ARG, "bad job list");
    if (njobs == 0) return SAGMS_OK;
    for (int i = 0; i < njobs; ++i) {
        if (!jobs[i].code) return fail(SAGMS_ERR_ARG, "job %d: code is NULL", i);
        const int rc = sagms_check_params(&jobs[i].params);
        if (rc != SAGMS_OK) return rc;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    // Library streams of this host thread (created once per thread and device): the jobs fork
    // from the caller's stream onto them and join back, so the call is capturable as one graph.
    constexpr int kSide = 8;
    thread_local std::vector<cudaStream_t> side[kMaxDevices];
    if (dev >= kMaxDevices) return fail(SAGMS_ERR_ARG, "device ordinal %d out of range", dev);
    while ((int)side[dev].size() < kSide) {
        cudaStream_t st;
        ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamCreate");
        side[dev].push_back(st);
    }
    const int used = std::min(njobs, kSide);
    std::vector<cudaEvent_t> ev(used + 1, nullptr);
    for (auto& e : ev) {
        ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (ce != cudaSuccess) {
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            return cuda_fail(ce, "cudaEventCreate");
        }
    }
    int rc = SAGMS_OK;
    ce = cudaEventRecord(ev[0], stream);
    for (int k = 0; k < used && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(side[dev][k], ev[0], 0);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "multi fork");
    for (int i = 0; i < njobs && rc == SAGMS_OK; ++i) {
        const sagms_job& j = jobs[i];
        rc = launch_decode(j.code, &j.params, j.shots, j.d_syn, j.d_L0, j.d_err, j.d_conv, j.d_iters, nullptr,
                           side[dev][i % kSide]);
    }
    for (int k = 0; k < used; ++k) {
        cudaEventRecord(ev[k + 1], side[dev][k]);
        cudaStreamWaitEvent(stream, ev[k + 1], 0);
    }
    for (auto& e : ev) cudaEventDestroy(e);
    ce = cudaGetLastError();
    if (rc == SAGMS_OK && ce != cudaSuccess) rc = cuda_fail(ce, "multi join");
    return rc;
}

struct sagms_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

int sagms_graph_create(const sagms_job* jobs, int32_t njobs, sagms_graph** out) {
    if (!out) return fail(SAGMS_ERR_ARG, "out is NULL");
    *out = nullptr;
    cudaStream_t st;
    cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamCreate");
    ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) { cudaStreamDestroy(st); return cuda_fail(ce, "begin capture"); }
    int rc = sagms_decode_multi(jobs, njobs, st);
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(st, &g);
    cudaStreamDestroy(st);
    if (rc != SAGMS_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
    cudaGraphExec_t ex = nullptr;
    ce = cudaGraphInstantiate(&ex, g, 0);
    if (ce != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ce, "graph instantiate"); }
    *out = new sagms_graph{g, ex};
    return SAGMS_OK;
}

int sagms_graph_launch(sagms_graph* g, void* stream) {
    if (!g) return fail(SAGMS_ERR_ARG, "graph is NULL");
    const cudaError_t ce = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
    return ce == cudaSuccess ? SAGMS_OK : cuda_fail(ce, "graph launch");
}

void sagms_graph_destroy(sagms_graph* g) {
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}

}  // extern "C"
