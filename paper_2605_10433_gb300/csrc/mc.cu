// Fused Monte Carlo frame-error estimation (include/sagms.h, "Fused Monte Carlo"): frame
// sampling and syndrome formation, the logical check, and the batch loop of the simulation
// protocol of Sec. V (setup), all on the GPU around the decoder of sagms.cu.
//
// Sampler.  Frame t of key `seed` is the flip pattern of the counter-based generator
// described in include/sagms.h (Philox4x32-10 blocks, geometric gaps looked up in the table
// T[g] = floor((1 - q)^g 2^32)).  Draw d gives a gap g_d; the flipped positions are
// pos_k = sum_{i <= k} (g_i + 1) - 1 for every k with pos_k < n.  A warp draws 32
// consecutive gaps at once (one per lane, each lane computing its own Philox block), turns
// them into positions with an inclusive warp scan, and repeats until a position reaches n.
// Pattern and syndrome of the frame are assembled in the warp's shared-memory slice and
// written out coalesced.
//
// Check.  A converged frame with residual r = e XOR e_hat fails when x . r = 1 (mod 2) for
// an attached X-logical x: H_X r = 0 puts r in ker(H_X) = rowspace(H_Z) + span(Z-logicals),
// and r is in rowspace(H_Z) = ker(H_Z)^perp exactly when it is orthogonal to ker(H_Z) =
// rowspace(H_X) + span(X-logicals), i.e. to the X-logicals.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/sagms.h"
#include "internal.h"

using sagms_internal::CodeView;

namespace {

constexpr int kMcThreads = 256;   // 8 warps per CTA, one frame per warp at a time
constexpr uint32_t kCtrTag = 0x53414721u;

int mc_fail(int code, const char* msg) { return sagms_internal::set_error(code, msg); }

// ---------------------------------------------------------------------------------------
// Host: the geometric-gap table and the logical basis.

// T[g] for g = 0..n: T[0] = 2^32 - 1 ("always"), then floor((1 - q)^g 2^32) with the powers
// formed by repeated double multiplication, 2^32 - 1 where that reaches 2^32 and 0 below 1.
std::vector<uint32_t> gap_table(double q, int n) {
    std::vector<uint32_t> T((size_t)n + 1);
    const double two32 = 4294967296.0;
    double pw = 1.0;
    for (int g = 0; g <= n; ++g) {
        const double t = pw * two32;
        T[g] = (g == 0 || t >= two32) ? 0xFFFFFFFFu : (t < 1.0 ? 0u : (uint32_t)t);
        pw *= (1.0 - q);
    }
    return T;
}

using Row = std::vector<uint64_t>;

bool csr_rows(int32_t n, int32_t m, const int32_t* rp, const int32_t* ci, std::vector<Row>* out) {
    if (m < 0 || (m > 0 && (!rp || (rp[m] > 0 && !ci))) || (m > 0 && rp[0] != 0)) return false;
    const size_t words = ((size_t)n + 63) / 64;
    out->assign((size_t)m, Row(words, 0));
    for (int32_t i = 0; i < m; ++i) {
        if (rp[i + 1] < rp[i]) return false;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = ci[e];
            if (j < 0 || j >= n) return false;
            (*out)[i][j >> 6] ^= 1ull << (j & 63);
        }
    }
    return true;
}

int lowest_bit(const Row& r) {
    for (size_t w = 0; w < r.size(); ++w)
        if (r[w]) return (int)(w * 64 + __builtin_ctzll(r[w]));
    return -1;
}

void xor_into(Row& a, const Row& b) {
    for (size_t w = 0; w < a.size(); ++w) a[w] ^= b[w];
}

// Echelon basis keyed by pivot (the lowest set bit of each basis row, all distinct).
// reduce(r) XORs into r the basis row of every pivot it meets, scanning bits upward (a basis
// row only has bits at or above its pivot); insert adds a row that does not reduce to zero.
struct Echelon {
    std::vector<int> pivot_of_col;   // column -> basis index, -1
    std::vector<Row> rows;
    explicit Echelon(int n) : pivot_of_col((size_t)n, -1) {}
    void reduce(Row& r) const {
        for (size_t w = 0; w < r.size(); ++w) {
            uint64_t seen = 0;
            while (const uint64_t x = r[w] & ~seen) {
                const uint64_t low = x & (~x + 1);
                const int b = pivot_of_col[w * 64 + __builtin_ctzll(x)];
                if (b >= 0) xor_into(r, rows[b]);
                seen |= low;
            }
        }
    }
    bool insert(Row r) {
        reduce(r);
        const int c = lowest_bit(r);
        if (c < 0) return false;
        pivot_of_col[c] = (int)rows.size();
        rows.push_back(std::move(r));
        return true;
    }
};

// Basis of ker(H) for H given as rows: reduced row echelon form, one vector per free column.
std::vector<Row> kernel_basis(int n, std::vector<Row> H) {
    const size_t words = ((size_t)n + 63) / 64;
    std::vector<int> pivot_cols;
    size_t rank = 0;
    for (int c = 0; c < n && rank < H.size(); ++c) {
        size_t piv = rank;
        while (piv < H.size() && !((H[piv][c >> 6] >> (c & 63)) & 1ull)) ++piv;
        if (piv == H.size()) continue;
        std::swap(H[rank], H[piv]);
        for (size_t i = 0; i < H.size(); ++i)
            if (i != rank && ((H[i][c >> 6] >> (c & 63)) & 1ull)) xor_into(H[i], H[rank]);
        pivot_cols.push_back(c);
        ++rank;
    }
    std::vector<char> is_pivot((size_t)n, 0);
    for (int c : pivot_cols) is_pivot[c] = 1;
    std::vector<Row> out;
    for (int f = 0; f < n; ++f) {
        if (is_pivot[f]) continue;
        Row x(words, 0);
        x[f >> 6] |= 1ull << (f & 63);
        for (size_t r = 0; r < pivot_cols.size(); ++r)
            if ((H[r][f >> 6] >> (f & 63)) & 1ull) x[pivot_cols[r] >> 6] |= 1ull << (pivot_cols[r] & 63);
        out.push_back(std::move(x));
    }
    return out;
}

// ---------------------------------------------------------------------------------------
// Device.

// One Philox4x32-10 block (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the two
// 32 x 32 -> 64-bit products with multipliers 0xD2511F53 and 0xCD9E8D57, the key advanced
// by the Weyl increments 0x9E3779B9 and 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Largest g in [0, n] with u < T[g] (T non-increasing, T[0] = 2^32 - 1; g = 0 when u >= T[1]).
__device__ __forceinline__ int gap_of(const uint32_t* __restrict__ T, int n, uint32_t u) {
    if (u >= __ldg(T + 1)) return 0;
    int lo = 1, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (u < __ldg(T + mid)) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kMcThreads) mc_sample_kernel(
    int m, int n, const uint16_t* __restrict__ qchk, int dv, const uint32_t* __restrict__ T, int flips,
    uint32_t k0, uint32_t k1, unsigned long long shot0, long long shots, float L0, uint32_t* err, uint32_t* syn,
    float* L0out) {
    extern __shared__ uint32_t mc_sh[];
    const int nw = (n + 31) >> 5, mw = (m + 31) >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = kMcThreads / 32;
    uint32_t* e = mc_sh + warp * (nw + mw);
    uint32_t* s = e + nw;
    for (long long t = (long long)blockIdx.x * wpb + warp; t < shots; t += (long long)gridDim.x * wpb) {
        for (int w = lane; w < nw + mw; w += 32) e[w] = 0u;
        __syncwarp();
        if (flips) {
            const unsigned long long shot = shot0 + (unsigned long long)t;
            int base = 0;        // position where the next gap starts
            uint32_t d0 = 0;     // first draw of this round
            while (true) {
                const uint32_t d = d0 + (uint32_t)lane;
                const uint4 b = philox4x32_10(make_uint4(d >> 2, (uint32_t)shot, (uint32_t)(shot >> 32), kCtrTag), k0, k1);
                const uint32_t sel = d & 3u;
                const uint32_t u = sel == 0 ? b.x : (sel == 1 ? b.y : (sel == 2 ? b.z : b.w));
                int a = gap_of(T, n, u) + 1;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, a, o);
                    if (lane >= o) a += y;
                }
                const int pos = base + a - 1;
                if (pos < n) {
                    atomicOr(&e[pos >> 5], 1u << (pos & 31));
                    for (int q = 0; q < dv; ++q) {
                        const uint32_t r = __ldg(qchk + (size_t)q * n + pos);
                        if (r != 0xFFFFu) atomicXor(&s[r >> 5], 1u << (r & 31));
                    }
                }
                const int last = __shfl_sync(0xffffffffu, pos, 31);
                if (last >= n - 1) break;   // the next position is >= n
                base = last + 1;
                d0 += 32;
            }
        }
        __syncwarp();
        if (err)
            for (int w = lane; w < nw; w += 32) err[t * nw + w] = e[w];
        if (syn)
            for (int w = lane; w < mw; w += 32) syn[t * mw + w] = s[w];
        if (L0out && lane == 0) L0out[t] = L0;
        __syncwarp();
    }
}

// Per frame: 0 success, 1 not converged, 2 converged to a nontrivial logical.  Counts:
// [shots, failures, not_converged, logical, iters_sum], per CTA in shared memory, then added.
__global__ void __launch_bounds__(kMcThreads) mc_check_kernel(
    int n, int k, const uint32_t* __restrict__ L, long long shots, const uint32_t* __restrict__ err,
    const uint32_t* __restrict__ ehat, const uint8_t* __restrict__ conv, const int32_t* __restrict__ iters,
    uint8_t* fail, unsigned long long* counts) {
    __shared__ unsigned long long c[5];
    if (threadIdx.x < 5) c[threadIdx.x] = 0ull;
    __syncthreads();
    const int nw = (n + 31) >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = kMcThreads / 32;
    unsigned long long mine[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
    for (long long t = (long long)blockIdx.x * wpb + warp; t < shots; t += (long long)gridDim.x * wpb) {
        int f = 0;
        if (!conv[t]) {
            f = 1;
        } else {
            // 32 logicals at a time: bit j of par = parity of x_j . r accumulated over words
            for (int j0 = 0; j0 < k && f == 0; j0 += 32) {
                uint32_t par = 0u;
                for (int w = lane; w < nw; w += 32) {
                    const uint32_t r = err[t * nw + w] ^ ehat[t * nw + w];
                    if (!r) continue;
                    const int jn = min(32, k - j0);
                    for (int j = 0; j < jn; ++j) par ^= (uint32_t)(__popc(__ldg(L + (size_t)(j0 + j) * nw + w) & r) & 1) << j;
                }
                if (__reduce_xor_sync(0xffffffffu, par)) f = 2;
            }
        }
        if (lane == 0) {
            mine[0] += 1;
            mine[1] += f != 0;
            mine[2] += f == 1;
            mine[3] += f == 2;
            mine[4] += (unsigned long long)max(iters[t], 0);
            if (fail) fail[t] = (uint8_t)f;
        }
    }
    if (lane == 0)
        for (int i = 0; i < 5; ++i)
            if (mine[i]) atomicAdd(&c[i], mine[i]);
    __syncthreads();
    if (threadIdx.x < 5 && c[threadIdx.x]) atomicAdd(counts + threadIdx.x, c[threadIdx.x]);
}

int grid_for(long long shots, int dev) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (shots + kMcThreads / 32 - 1) / (kMcThreads / 32);
    return (int)std::max(1LL, std::min(want, (long long)std::max(sms, 1) * 8));
}

// Checks that the current device is the code's.
int on_code_device(const CodeView& v) {
    int dev = 0;
    const cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "cudaGetDevice");
    if (dev != v.device) return mc_fail(SAGMS_ERR_ARG, "code was loaded on another device");
    return SAGMS_OK;
}

bool misaligned(const void* ptr, uintptr_t bytes) { return (reinterpret_cast<uintptr_t>(ptr) & (bytes - 1)) != 0; }

int sample_launch(const CodeView& v, uint64_t seed, double q, float L0, int64_t shot0, int64_t shots,
                  const uint32_t* d_T, uint32_t* d_err, uint32_t* d_syn, float* d_L0, cudaStream_t st) {
    const size_t smem = (size_t)(kMcThreads / 32) * (((v.n + 31) / 32) + ((v.m + 31) / 32)) * 4;
    const void* fn = reinterpret_cast<const void*>(mc_sample_kernel);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, v.device);
    if (smem > (size_t)optin) return mc_fail(SAGMS_ERR_SIZE, "code too large for the sampler's shared memory");
    cudaError_t ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "cudaFuncSetAttribute");
    mc_sample_kernel<<<grid_for(shots, v.device), kMcThreads, smem, st>>>(
        v.m, v.n, v.d_qchk, v.dv_max, d_T, q > 0.0 ? 1 : 0, (uint32_t)seed, (uint32_t)(seed >> 32),
        (unsigned long long)shot0, (long long)shots, L0, d_err, d_syn, d_L0);
    ce = cudaGetLastError();
    return ce == cudaSuccess ? SAGMS_OK : sagms_internal::cuda_error(ce, "sampler launch");
}

int check_launch(const CodeView& v, int64_t shots, const uint32_t* d_err, const uint32_t* d_ehat,
                 const uint8_t* d_conv, const int32_t* d_iters, uint8_t* d_fail, sagms_mc_counts* d_counts,
                 cudaStream_t st) {
    mc_check_kernel<<<grid_for(shots, v.device), kMcThreads, 0, st>>>(
        v.n, v.k_logicals, v.d_logicals, (long long)shots, d_err, d_ehat, d_conv, d_iters, d_fail,
        reinterpret_cast<unsigned long long*>(d_counts));
    const cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? SAGMS_OK : sagms_internal::cuda_error(ce, "check launch");
}

}  // namespace

extern "C" {

int sagms_x_logicals(int32_t n, int32_t mx, const int32_t* hx_row_ptr, const int32_t* hx_col_idx, int32_t mz,
                     const int32_t* hz_row_ptr, const int32_t* hz_col_idx, int32_t max_k, uint32_t* logicals,
                     int32_t* k) {
    if (!k || n < 1 || max_k < 0 || (max_k > 0 && !logicals)) return mc_fail(SAGMS_ERR_ARG, "bad arguments");
    std::vector<Row> HX, HZ;
    if (!csr_rows(n, mx, hx_row_ptr, hx_col_idx, &HX)) return mc_fail(SAGMS_ERR_CSR, "malformed H_X");
    if (!csr_rows(n, mz, hz_row_ptr, hz_col_idx, &HZ)) return mc_fail(SAGMS_ERR_CSR, "malformed H_Z");
    for (const Row& x : HX)
        for (const Row& z : HZ) {
            int par = 0;
            for (size_t w = 0; w < x.size(); ++w) par ^= __builtin_popcountll(x[w] & z[w]) & 1;
            if (par) return mc_fail(SAGMS_ERR_PARAM, "H_X H_Z^T != 0: not a CSS pair");
        }
    Echelon basis(n);
    for (const Row& x : HX) basis.insert(x);
    const std::vector<Row> ker = kernel_basis(n, HZ);
    std::vector<Row> found;
    for (const Row& x : ker)
        if (basis.insert(x)) found.push_back(x);
    *k = (int32_t)found.size();
    const int nw = (n + 31) / 32;
    for (int32_t j = 0; j < std::min<int32_t>(max_k, *k); ++j)
        for (int w = 0; w < nw; ++w) logicals[(size_t)j * nw + w] = (uint32_t)(found[j][w / 2] >> (32 * (w % 2)));
    return SAGMS_OK;
}

int sagms_mc_set_logicals(sagms_code* code, int32_t k, const uint32_t* logicals) {
    if (!code) return mc_fail(SAGMS_ERR_ARG, "code is NULL");
    if (k < 0 || (k > 0 && !logicals)) return mc_fail(SAGMS_ERR_ARG, "bad logical operators");
    const CodeView v = sagms_internal::code_view(code);
    const int rc = on_code_device(v);
    if (rc != SAGMS_OK) return rc;
    return sagms_internal::attach_logicals(code, k, logicals);
}

int sagms_mc_sample(const sagms_code* code, uint64_t seed, double q, float L0, int64_t shot0, int64_t shots,
                    uint32_t* d_err, uint32_t* d_syn, float* d_L0, void* stream) {
    if (!(q >= 0.0 && q < 1.0)) return mc_fail(SAGMS_ERR_PARAM, "flip probability outside [0, 1)");
    if (shots < 0 || shot0 < 0) return mc_fail(SAGMS_ERR_ARG, "negative shot range");
    // each output is optional; those given take 4-byte words
    if (misaligned(d_err, 4) || misaligned(d_syn, 4) || misaligned(d_L0, 4))
        return mc_fail(SAGMS_ERR_ARG, "device buffers must be 4-byte aligned");
    if (!code) return mc_fail(SAGMS_ERR_ARG, "code is NULL");
    if (shots == 0) return SAGMS_OK;
    const CodeView v = sagms_internal::code_view(code);
    int rc = on_code_device(v);
    if (rc != SAGMS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::vector<uint32_t> T = gap_table(q, v.n);
    uint32_t* d_T = nullptr;
    cudaError_t ce = cudaMallocAsync(reinterpret_cast<void**>(&d_T), T.size() * 4, st);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "gap table allocation");
    // From pageable host memory the copy is staged before the call returns, so the table
    // may go out of scope afterwards.
    ce = cudaMemcpyAsync(d_T, T.data(), T.size() * 4, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
        cudaFreeAsync(d_T, st);
        return sagms_internal::cuda_error(ce, "gap table upload");
    }
    rc = sample_launch(v, seed, q, L0, shot0, shots, d_T, d_err, d_syn, d_L0, st);
    cudaFreeAsync(d_T, st);
    return rc;
}

int sagms_mc_check(const sagms_code* code, int64_t shots, const uint32_t* d_err, const uint32_t* d_err_hat,
                   const uint8_t* d_conv, const int32_t* d_iters, uint8_t* d_fail, sagms_mc_counts* d_counts,
                   void* stream) {
    if (shots < 0) return mc_fail(SAGMS_ERR_ARG, "shots < 0");
    if (shots > 0) {
        if (!d_err || !d_err_hat || !d_conv || !d_iters || !d_counts)
            return mc_fail(SAGMS_ERR_ARG, "NULL device buffer");
        // 4-byte words and counts; the counters are 64-bit atomics
        if (misaligned(d_err, 4) || misaligned(d_err_hat, 4) || misaligned(d_iters, 4) || misaligned(d_counts, 8))
            return mc_fail(SAGMS_ERR_ARG, "device buffers misaligned (4-byte words, 8-byte counters)");
    }
    if (!code) return mc_fail(SAGMS_ERR_ARG, "code is NULL");
    if (shots == 0) return SAGMS_OK;
    const CodeView v = sagms_internal::code_view(code);
    if (v.k_logicals < 0) return mc_fail(SAGMS_ERR_ARG, "no logical operators attached (sagms_mc_set_logicals)");
    const int rc = on_code_device(v);
    if (rc != SAGMS_OK) return rc;
    return check_launch(v, shots, d_err, d_err_hat, d_conv, d_iters, d_fail, d_counts, static_cast<cudaStream_t>(stream));
}

int sagms_mc_run(const sagms_code* code, const sagms_params* params, uint64_t seed, double q, float L0,
                 int64_t target_failures, int64_t max_shots, int64_t batch, sagms_mc_counts* counts) {
    if (!code || !counts) return mc_fail(SAGMS_ERR_ARG, "NULL argument");
    int rc = sagms_check_params(params);
    if (rc != SAGMS_OK) return rc;
    if (params->flags & SAGMS_FLAG_L0_PER_QUBIT) return mc_fail(SAGMS_ERR_ARG, "the Monte Carlo run uses a per-frame prior");
    if (!(q >= 0.0 && q < 1.0)) return mc_fail(SAGMS_ERR_PARAM, "flip probability outside [0, 1)");
    if (batch < 1 || max_shots < 0 || target_failures < 0) return mc_fail(SAGMS_ERR_ARG, "bad run limits");
    const CodeView v = sagms_internal::code_view(code);
    if (v.k_logicals < 0) return mc_fail(SAGMS_ERR_ARG, "no logical operators attached (sagms_mc_set_logicals)");
    rc = on_code_device(v);
    if (rc != SAGMS_OK) return rc;
    if (counts->failures >= target_failures || counts->shots >= max_shots) return SAGMS_OK;
    const int64_t B = std::min(batch, max_shots - counts->shots);
    const size_t nw = (size_t)(v.n + 31) / 32, mw = (size_t)(v.m + 31) / 32;

    cudaStream_t st = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "cudaStreamCreate");
    const std::vector<uint32_t> T = gap_table(q, v.n);
    uint32_t *d_T = nullptr, *d_err = nullptr, *d_syn = nullptr, *d_ehat = nullptr;
    float* d_L0 = nullptr;
    uint8_t* d_conv = nullptr;
    int32_t* d_iters = nullptr;
    sagms_mc_counts* d_counts = nullptr;
    ce = cudaMallocAsync(reinterpret_cast<void**>(&d_T), T.size() * 4, st);
    if (ce == cudaSuccess) ce = cudaMallocAsync(reinterpret_cast<void**>(&d_err), (size_t)B * nw * 4, st);
    if (ce == cudaSuccess) ce = cudaMallocAsync(reinterpret_cast<void**>(&d_syn), (size_t)B * mw * 4, st);
    if (ce == cudaSuccess) ce = cudaMallocAsync(reinterpret_cast<void**>(&d_ehat), (size_t)B * nw * 4, st);
    if (ce == cudaSuccess) ce = cudaMallocAsync(reinterpret_cast<void**>(&d_L0), (size_t)B * 4, st);
    if (ce == cudaSuccess) ce = cudaMallocAsync(reinterpret_cast<void**>(&d_conv), (size_t)B, st);
    if (ce == cudaSuccess) ce = cudaMallocAsync(reinterpret_cast<void**>(&d_iters), (size_t)B * 4, st);
    if (ce == cudaSuccess) ce = cudaMallocAsync(reinterpret_cast<void**>(&d_counts), sizeof(sagms_mc_counts), st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_T, T.data(), T.size() * 4, cudaMemcpyHostToDevice, st);
    rc = ce == cudaSuccess ? SAGMS_OK : sagms_internal::cuda_error(ce, "Monte Carlo buffers");
    while (rc == SAGMS_OK && counts->failures < target_failures && counts->shots < max_shots) {
        const int64_t b = std::min(B, max_shots - counts->shots);
        const sagms_internal::NvtxRange nvtx("sagms_mc_batch");
        sagms_mc_counts h = {0, 0, 0, 0, 0};
        ce = cudaMemsetAsync(d_counts, 0, sizeof(sagms_mc_counts), st);
        if (ce != cudaSuccess) { rc = sagms_internal::cuda_error(ce, "counter reset"); break; }
        rc = sample_launch(v, seed, q, L0, counts->shots, b, d_T, d_err, d_syn, d_L0, st);
        if (rc == SAGMS_OK) rc = sagms_internal::launch(code, params, b, d_syn, d_L0, d_ehat, d_conv, d_iters, st, nullptr);
        if (rc == SAGMS_OK) rc = check_launch(v, b, d_err, d_ehat, d_conv, d_iters, nullptr, d_counts, st);
        if (rc != SAGMS_OK) break;
        ce = cudaMemcpyAsync(&h, d_counts, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc = sagms_internal::cuda_error(ce, "Monte Carlo batch"); break; }
        counts->shots += h.shots;
        counts->failures += h.failures;
        counts->not_converged += h.not_converged;
        counts->logical += h.logical;
        counts->iters_sum += h.iters_sum;
    }
    void* bufs[] = {d_T, d_err, d_syn, d_ehat, d_L0, d_conv, d_iters, d_counts};
    for (void* p : bufs)
        if (p) cudaFreeAsync(p, st);
    ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess && rc == SAGMS_OK) rc = sagms_internal::cuda_error(ce, "Monte Carlo teardown");
    cudaStreamDestroy(st);
    return rc;
}

}  // extern "C"
