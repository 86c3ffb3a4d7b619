// Quaternary (GF(4)) decoding: code loading and launches of gf4_kernel (gf4_kernel.cuh, any
// stabilizer matrix) and gf4_css_kernel (gf4_css_kernel.cuh, CSS matrices).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "gf4_css_kernel.cuh"
#include "gf4_kernel.cuh"
#include "internal.h"
#include "sagms.h"

using sagms::DecodeArgs;
using sagms::Gf4Layout;

namespace {

int gfail(int code, const char* msg) { return sagms_internal::set_error(code, msg); }

// Compiled shapes: padded check degree DC and qubit degree DV (a CSS matrix of weight-w GB
// codes has both equal to 2w); a code takes the first that covers its largest degrees.
struct Gf4Variant {
    int dc, dv;
    void (*fn[2])(const DecodeArgs, const Gf4Layout);   // MS family, BP
};
#define SAGMS_GF4(DC, DV) \
    Gf4Variant { DC, DV, {sagms::gf4_kernel<DC, DV, false>, sagms::gf4_kernel<DC, DV, true>} }
const Gf4Variant kGf4Variants[] = {SAGMS_GF4(6, 6), SAGMS_GF4(8, 8), SAGMS_GF4(10, 10), SAGMS_GF4(12, 12),
                                   SAGMS_GF4(16, 16)};
#undef SAGMS_GF4
constexpr int kNumGf4 = sizeof(kGf4Variants) / sizeof(kGf4Variants[0]);

// Column-indexed CSS shapes: DC check slots, DH message rows per row type (DC = 2 DH); a code
// takes the first that covers its check degree and its largest per-type qubit degree.
struct Gf4CssVariant {
    int dc, dh;
    void (*fn[2])(const DecodeArgs, const uint32_t*);   // MS family, BP
};
#define SAGMS_GF4_CSS(DC, DH) \
    Gf4CssVariant { DC, DH, {sagms::gf4_css_kernel<DC, DH, false>, sagms::gf4_css_kernel<DC, DH, true>} }
const Gf4CssVariant kGf4CssVariants[] = {SAGMS_GF4_CSS(6, 3), SAGMS_GF4_CSS(8, 4), SAGMS_GF4_CSS(10, 5),
                                         SAGMS_GF4_CSS(12, 6), SAGMS_GF4_CSS(16, 8)};
#undef SAGMS_GF4_CSS
constexpr int kNumGf4Css = sizeof(kGf4CssVariants) / sizeof(kGf4CssVariants[0]);

}  // namespace

struct sagms_gf4_code {
    int m, n, nnz, dc_max, dv_max, variant, Mp, Np, device;
    uint32_t pauli_set;   // bit P: the matrix has an entry of Pauli P (1 X, 2 Z, 3 Y)
    uint16_t* d_colT;
    uint32_t* d_vneT;
    int css_variant;      // column-indexed CSS shape, or -1 (not CSS, or no slot assignment)
    uint32_t* d_colS;     // [DC][Mp] biased byte offsets of the CSS kernel
};

namespace {

// The column-indexed layout of a CSS matrix (every row all X or all Z): per row type, the slot
// assignment sagms_column_slots would give that type's rows (distinct mod DH among each
// qubit's edges of the type), then the biased byte offsets colS[j][i] = 4 col + (type Z ?
// half : 0); padded slots and checks past m point at the padding column n of the X half.
// Returns the shape, or -1 (the generic kernel then decodes the matrix).
int css_layout(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* pauli, int dc_max,
               int Mp, int Np, std::vector<uint32_t>& colS) {
    std::vector<int> type(m, 0);
    for (int i = 0; i < m; ++i) {
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (pauli[e] == 3 || (type[i] != 0 && type[i] != pauli[e])) return -1;
            type[i] = pauli[e];
        }
    }
    std::vector<int> dvt[2] = {std::vector<int>(n, 0), std::vector<int>(n, 0)};
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) dvt[type[i] == 2][col_idx[e]]++;
    int dh_need = 1;
    for (int h = 0; h < 2; ++h) dh_need = std::max(dh_need, *std::max_element(dvt[h].begin(), dvt[h].end()));
    int var = -1;
    for (int v = 0; v < kNumGf4Css && var < 0; ++v)
        if (kGf4CssVariants[v].dc >= dc_max && kGf4CssVariants[v].dh >= dh_need) var = v;
    if (var < 0) return -1;
    const int DC = kGf4CssVariants[var].dc, DH = kGf4CssVariants[var].dh;
    const uint32_t half = (uint32_t)sagms::gf4_css_half_bytes(DH, Np);
    colS.assign((size_t)DC * Mp, (uint32_t)n * 4u);
    for (int h = 0; h < 2; ++h) {
        // this type's rows as their own CSR (rows without edges count as X rows and stay padded)
        std::vector<int> rows;
        std::vector<int32_t> rp(1, 0), ci;
        for (int i = 0; i < m; ++i) {
            if ((type[i] == 2) != (h == 1)) continue;
            rows.push_back(i);
            for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) ci.push_back(col_idx[e]);
            rp.push_back((int32_t)ci.size());
        }
        if (rows.empty()) continue;
        // degrees within the shape: qubit degree of this type <= DH, row degree <= DC = 2 DH
        const std::vector<int> slot =
            sagms_internal::column_slot_assignment((int)rows.size(), n, rp.data(), ci.data(), DH);
        if (slot.size() != ci.size()) return -1;
        for (size_t r = 0; r < rows.size(); ++r)
            for (int e = rp[r]; e < rp[r + 1]; ++e) {
                if (slot[e] < 0 || slot[e] >= DC) return -1;
                colS[(size_t)slot[e] * Mp + rows[r]] = (uint32_t)ci[e] * 4u + (h ? half : 0u);
            }
    }
    return var;
}

}  // namespace

extern "C" {

int sagms_gf4_load_code(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                        const uint8_t* pauli, sagms_gf4_code** out) {
    if (!out) return gfail(SAGMS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (m < 1 || m > 512 || n < 1 || n > 16382 || nnz < 0 || !row_ptr || (nnz > 0 && (!col_idx || !pauli)))
        return gfail(SAGMS_ERR_ARG, "need 1 <= m <= 512 checks, 1 <= n <= 16382 qubits and the CSR arrays");
    if (row_ptr[0] != 0 || row_ptr[m] != nnz) return gfail(SAGMS_ERR_CSR, "row_ptr must run from 0 to nnz");
    std::vector<int> dv(n, 0);
    int dc_max = 0;
    uint32_t pauli_set = 0;
    for (int i = 0; i < m; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return gfail(SAGMS_ERR_CSR, "row_ptr decreases");
        dc_max = std::max(dc_max, row_ptr[i + 1] - row_ptr[i]);
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (col_idx[e] < 0 || col_idx[e] >= n) return gfail(SAGMS_ERR_CSR, "column out of range");
            if (pauli[e] < 1 || pauli[e] > 3) return gfail(SAGMS_ERR_CSR, "Pauli entries must be 1 (X), 2 (Z) or 3 (Y)");
            for (int f = row_ptr[i]; f < e; ++f)
                if (col_idx[f] == col_idx[e]) return gfail(SAGMS_ERR_CSR, "duplicate column in a row");
            dv[col_idx[e]]++;
            pauli_set |= 1u << pauli[e];
        }
    }
    const int dv_max = *std::max_element(dv.begin(), dv.end());
    int variant = -1;
    for (int v = 0; v < kNumGf4; ++v)
        if (kGf4Variants[v].dc >= dc_max && kGf4Variants[v].dv >= dv_max) { variant = v; break; }
    if (variant < 0) return gfail(SAGMS_ERR_DEGREE, "check or qubit degree above 16");
    const int DC = kGf4Variants[variant].dc, DV = kGf4Variants[variant].dv;
    const int Mp = std::max(32, (m + 31) / 32 * 32), Np = (n + 1 + 31) / 32 * 32;
    // slot-major edges; a padded slot points at column n with Pauli 0
    std::vector<uint16_t> colT((size_t)DC * Mp, (uint16_t)n);
    std::vector<uint32_t> vneT((size_t)DV * Np, (uint32_t)(DC * Mp));   // zero slot, Pauli 0
    std::vector<int> fill(n, 0);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int j = e - row_ptr[i], c = col_idx[e];
            colT[(size_t)j * Mp + i] = (uint16_t)(c | (pauli[e] << 14));
            vneT[(size_t)fill[c]++ * Np + c] = (uint32_t)(j * Mp + i) | ((uint32_t)pauli[e] << 16);
        }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "cudaGetDevice");
    std::vector<uint32_t> colS;
    const int css = css_layout(m, n, row_ptr, col_idx, pauli, dc_max, Mp, Np, colS);
    sagms_gf4_code* code = new sagms_gf4_code();
    code->m = m; code->n = n; code->nnz = (int)nnz; code->dc_max = dc_max; code->dv_max = dv_max;
    code->variant = variant; code->Mp = Mp; code->Np = Np; code->device = dev; code->pauli_set = pauli_set;
    code->d_colT = nullptr; code->d_vneT = nullptr; code->css_variant = css; code->d_colS = nullptr;
    ce = cudaMalloc(reinterpret_cast<void**>(&code->d_colT), colT.size() * sizeof(uint16_t));
    if (ce == cudaSuccess) ce = cudaMalloc(reinterpret_cast<void**>(&code->d_vneT), vneT.size() * sizeof(uint32_t));
    if (ce == cudaSuccess && css >= 0) ce = cudaMalloc(reinterpret_cast<void**>(&code->d_colS), colS.size() * 4);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(code->d_colT, colT.data(), colT.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(code->d_vneT, vneT.data(), vneT.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && css >= 0)
        ce = cudaMemcpy(code->d_colS, colS.data(), colS.size() * 4, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        cudaFree(code->d_colT);
        cudaFree(code->d_vneT);
        cudaFree(code->d_colS);
        delete code;
        return sagms_internal::cuda_error(ce, "sagms_gf4_load_code upload");
    }
    *out = code;
    return SAGMS_OK;
}

void sagms_gf4_free_code(sagms_gf4_code* code) {
    if (!code) return;
    cudaFree(code->d_colT);
    cudaFree(code->d_vneT);
    cudaFree(code->d_colS);
    delete code;
}

int sagms_gf4_decode_trace(const sagms_gf4_code* code, const sagms_params* p, int64_t shots, const uint32_t* d_syn,
                           const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, float* d_trace,
                           void* stream_v) {
    const sagms_internal::NvtxRange nvtx("sagms_gf4_decode");
    if (!code) return gfail(SAGMS_ERR_ARG, "code is NULL");
    int rc = sagms_check_params(p);
    if (rc != SAGMS_OK) return rc;
    if (p->flags & ~(uint32_t)(SAGMS_FLAG_NO_EARLY_STOP | SAGMS_FLAG_GENERIC_KERNEL))
        return gfail(SAGMS_ERR_PARAM, "the GF(4) decoder takes one prior per shot and no flag but "
                                      "SAGMS_FLAG_NO_EARLY_STOP and SAGMS_FLAG_GENERIC_KERNEL");
    if (shots < 0) return gfail(SAGMS_ERR_ARG, "shots < 0");
    if (shots == 0) return SAGMS_OK;
    if (!d_syn || !d_L0 || !d_err || !d_conv || !d_iters) return gfail(SAGMS_ERR_ARG, "NULL device buffer");
    auto al4 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 3u) == 0; };
    if (!al4(d_syn) || !al4(d_L0) || !al4(d_err) || !al4(d_iters) || (d_trace && !al4(d_trace)))
        return gfail(SAGMS_ERR_ARG, "device buffers must be 4-byte aligned");
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "cudaGetDevice");
    if (dev != code->device) return gfail(SAGMS_ERR_ARG, "code was loaded on another device");
    DecodeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.m = code->m; a.n = code->n; a.Mp = code->Mp; a.Np = code->Np;
    a.mode = p->mode;
    a.alpha = p->alpha;
    a.amin = p->alpha_min;
    a.amax = p->alpha_max;
    a.eta = (p->eta_unsat == 0.0f) ? 1.10f : p->eta_unsat;
    a.inv_m = 1.0f / (float)code->m;
    a.dcmax = code->dc_max;
    a.max_iter = p->max_iter;
    a.flags = (p->flags & SAGMS_FLAG_NO_EARLY_STOP) | (code->pauli_set << sagms::kGf4PauliShift);
    a.shots = shots;
    a.syn = d_syn; a.L0 = d_L0; a.err = d_err; a.conv = d_conv; a.iters = d_iters; a.trace = d_trace;
    int smem_optin = 0, sms = 0;
    ce = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "device attributes");
    const int bp = p->mode == SAGMS_BP ? 1 : 0;
    if (code->css_variant >= 0 && !(p->flags & SAGMS_FLAG_GENERIC_KERNEL)) {
        // the column-indexed CSS kernel, when its two halves fit a CTA
        const Gf4CssVariant& cv = kGf4CssVariants[code->css_variant];
        const size_t smem = sagms::gf4_css_smem_bytes(cv.dh, code->Np);
        if (smem <= (size_t)smem_optin) {
            auto fn = cv.fn[bp];
            ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "cudaFuncSetAttribute");
            int per_sm = 0;
            ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, code->Mp, smem);
            if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "occupancy query");
            if (per_sm < 1) return gfail(SAGMS_ERR_SIZE, "kernel does not fit on an SM");
            const long long grid = std::min<long long>(shots, (long long)per_sm * sms);
            fn<<<(unsigned)grid, code->Mp, smem, static_cast<cudaStream_t>(stream_v)>>>(a, code->d_colS);
            ce = cudaGetLastError();
            return ce == cudaSuccess ? SAGMS_OK : sagms_internal::cuda_error(ce, "gf4 css decode launch");
        }
    }
    const Gf4Variant& v = kGf4Variants[code->variant];
    auto fn = v.fn[bp];
    const size_t smem = sagms::gf4_smem_bytes(v.dc, v.dv, code->Mp, code->Np);
    if (smem > (size_t)smem_optin) return gfail(SAGMS_ERR_SIZE, "code needs more shared memory than a CTA has");
    ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "cudaFuncSetAttribute");
    int per_sm = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, code->Mp, smem);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "occupancy query");
    if (per_sm < 1) return gfail(SAGMS_ERR_SIZE, "kernel does not fit on an SM");
    const long long grid = std::min<long long>(shots, (long long)per_sm * sms);
    const Gf4Layout lay{code->d_colT, code->d_vneT};
    fn<<<(unsigned)grid, code->Mp, smem, static_cast<cudaStream_t>(stream_v)>>>(a, lay);
    ce = cudaGetLastError();
    return ce == cudaSuccess ? SAGMS_OK : sagms_internal::cuda_error(ce, "gf4 decode launch");
}

int sagms_gf4_layout(const sagms_gf4_code* code) {
    if (!code) return gfail(SAGMS_ERR_ARG, "code is NULL");
    return code->css_variant >= 0 ? 1 : 0;
}

int sagms_gf4_decode(const sagms_gf4_code* code, const sagms_params* p, int64_t shots, const uint32_t* d_syn,
                     const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, void* stream) {
    return sagms_gf4_decode_trace(code, p, shots, d_syn, d_L0, d_err, d_conv, d_iters, nullptr, stream);
}

}  // extern "C"
