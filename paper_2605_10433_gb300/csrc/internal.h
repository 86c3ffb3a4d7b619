// Declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <vector>

#include "../../include/sagms.h"

namespace sagms_internal {

// NVTX range over a host-side step (decode launch, serving request, Monte Carlo batch): shows
// up in Nsight timelines; costs a function-pointer test when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// How a decode is launched.  kernel: 0 automatic, 1 one shot per CTA, 2 two-slot, 3 two-group,
// 4 two-group with column-indexed messages;
// ctas_per_sm: 0 = occupancy limit; chunk_lg: log2 shots per claimed chunk, 0 = automatic;
// max_grid: cap on the number of CTAs, 0 = none (a small grid keeps a launch from holding
// every SM, so concurrent launches share the GPU CTA by CTA).
struct Plan {
    int kernel = 0;
    int ctas_per_sm = 0;
    int chunk_lg = 0;
    long long max_grid = 0;
    int* work = nullptr;   // caller-owned chunk counters (>= one per launch chunk); null: allocate
};

// sagms_decode with an explicit launch plan (nullptr: the code's own plan).
int launch(const sagms_code* code, const sagms_params* params, int64_t shots, const uint32_t* d_syn,
           const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, cudaStream_t stream,
           const Plan* plan);

// What the Monte Carlo engine reads of a loaded code.
struct CodeView {
    int m, n, dv_max, device;
    const uint16_t* d_qchk;     // [dv_max][n]: checks of each qubit (0xFFFF past its degree)
    int k_logicals;             // -1: none attached
    const uint32_t* d_logicals; // [k][ceil(n/32)]
};
CodeView code_view(const sagms_code* code);
// Attach logical operators (device copy owned by the code handle).
int attach_logicals(sagms_code* code, int k, const uint32_t* h_logicals);

// Column-indexed slot of every edge of a CSR matrix for D message rows (what
// sagms_column_slots computes: the CSR order when it already gives each qubit distinct slots
// mod D, else an edge colouring), or empty when there is none.  The caller guarantees a valid
// CSR with qubit degrees <= D and row degrees <= 2 D.  Records no error, so a caller that only
// probes whether a layout exists leaves the last-error string alone.
std::vector<int> column_slot_assignment(int m, int n, const int32_t* row_ptr, const int32_t* col_idx, int D);

// Record `msg` as the calling thread's last error and return `code`.
int set_error(int code, const char* msg);
int cuda_error(cudaError_t e, const char* what);

}  // namespace sagms_internal
