/*
 * sagms.h -- C ABI of libsagms.so, a GB300 (sm_103a) batched syndrome decoder for
 * quantum LDPC codes: plain Min-Sum (MS), fixed-scale Min-Sum (SMS), syndrome-adaptive
 * gain Min-Sum (SAGMS) and the tanh-rule belief-propagation reference (BP).
 *
 * Method: "Syndrome Adaptive Gain Control for Min-Sum Decoding of Quantum LDPC Codes"
 * (arXiv 2605.10433).  Each call decodes a batch of independent shots: for every shot,
 * the flooding-schedule iteration of Algorithm 1 on the Tanner graph of a binary
 * parity-check matrix H (m checks, n qubits), with early termination once the residual
 * syndrome of Eq. 1 is zero.
 *
 * Conventions for every entry point:
 *   - Return value: SAGMS_OK (0) or a negative SAGMS_ERR_* code; the message of the
 *     last failure on the calling thread is sagms_last_error_string().
 *   - Host arrays passed in are read during the call and never kept; the caller keeps
 *     ownership.  Device pointers are caller-owned device memory (any allocator); the
 *     library never frees them and never synchronises the caller's stream unless the
 *     entry point says so.
 *   - Packed bit layout: bit k of a pattern is bit (k % 32) of uint32 word k / 32.
 *     A syndrome occupies ceil(m/32) words per shot, an error estimate ceil(n/32).
 *   - A code handle may be used from several host threads and streams at once.  Its
 *     decoding behaviour is fixed by sagms_load_code; sagms_set_plan (atomic) and
 *     sagms_mc_set_logicals (not concurrently with a Monte Carlo call on the handle) are
 *     the only mutations.
 */
#ifndef SAGMS_H
#define SAGMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Decoder forms (Sec. II and III). */
enum {
    SAGMS_MS = 0,    /* Eq. 4: CN output = (-1)^{s_i} prod sgn * min |.| */
    SAGMS_SMS = 1,   /* Eq. 4 times a fixed alpha in (0, 1] */
    SAGMS_SAGMS = 2, /* Eq. 8 with the per-shot, per-check gain of Eq. 7 */
    SAGMS_BP = 3     /* Eq. 3, the phi-domain (tanh) rule */
};

/* Flags of sagms_params.flags. */
enum {
    /* d_L0 holds n per-qubit priors shared by all shots (LLR units) instead of one
     * prior per shot.  Without it the MS family runs in L0-normalised units. */
    SAGMS_FLAG_L0_PER_QUBIT = 1u,
    /* Run exactly max_iter rounds even after the residual syndrome reaches zero. */
    SAGMS_FLAG_NO_EARLY_STOP = 2u,
    /* Use the one-shot-per-CTA kernel even where a faster kernel exists (cross-checks:
     * all kernels give bitwise identical results, BP included). */
    SAGMS_FLAG_GENERIC_KERNEL = 4u,
    /* SAGMS only, per-shot priors only: the gain ceiling of Corollary 1.  Each shot's
     * alpha_max is alpha*(|L0|, d_c) of Eq. 9 for its own prior L0 and the code's largest
     * check degree d_c (alpha* decreases in d_c, Prop. 1, so on an irregular code this is
     * the most conservative ceiling), clamped to [alpha_min, 1/eta_unsat]; a zero prior gets
     * alpha_min.  params.alpha_max is then ignored. */
    SAGMS_FLAG_AUTO_CEILING = 16u,
    /* MS family only (SAGMS, SMS, MS), check degrees <= 24: a layered (serial-check)
     * schedule in place of Algorithm 1's flooding one -- a different decoder, with its own
     * results.  The checks form layers that share no qubit (check i joins the smallest
     * layer used by no earlier check sharing a qubit with it); a round visits the layers in
     * increasing order, and each check computes its Eq. 2 inputs from the messages as they
     * stand, including those replaced earlier in the same round.  The gains of Eq. 7 come
     * from the residual at the start of each round, the stopping rule and outputs are those
     * of Algorithm 1, and d_iters counts rounds.  The plan's kernel choice does not apply. */
    SAGMS_FLAG_LAYERED = 32u
};

/* Status codes. */
enum {
    SAGMS_OK = 0,
    SAGMS_ERR_ARG = -1,     /* null pointer, negative size, unknown flag */
    SAGMS_ERR_CSR = -2,     /* malformed CSR (row_ptr not monotone, column out of range, duplicate) */
    SAGMS_ERR_DEGREE = -3,  /* check degree > SAGMS_MAX_DC or qubit degree > SAGMS_MAX_DV */
    SAGMS_ERR_PARAM = -4,   /* parameters outside the ranges of Eq. 7 and Sec. II */
    SAGMS_ERR_OOM = -5,     /* device allocation failed */
    SAGMS_ERR_CUDA = -6,    /* a CUDA runtime call failed (no device, launch failure, ...) */
    SAGMS_ERR_TIMEOUT = -7, /* a bounded wait ran out */
    SAGMS_ERR_BUSY = -8,    /* resource temporarily unavailable */
    SAGMS_ERR_SIZE = -9,    /* code too large for one CTA's shared memory / thread block */
    SAGMS_ERR_CANCELLED = -10 /* serving: the request was cancelled before it ran */
};

#define SAGMS_MAX_DC 32     /* largest check degree |M(i)| */
#define SAGMS_MAX_DV 16     /* largest qubit degree |N(j)| */
#define SAGMS_MAX_M 1024    /* one thread per check within a CTA */

typedef struct sagms_code sagms_code; /* opaque, library-owned */

/*
 * Decoder parameters.
 *   mode:       SAGMS_MS / SAGMS_SMS / SAGMS_SAGMS / SAGMS_BP.
 *   alpha:      SMS scale, 0 < alpha <= 1 (Eq. 4 and the SMS rule of Sec. II).
 *   alpha_min, alpha_max, eta_unsat: SAGMS gain of Eq. 7, with
 *               2^-20 <= alpha_min <= alpha_max <= 1, eta_unsat >= 1 and
 *               alpha_max * eta_unsat <= 1 (the stability constraint of Sec. III-A).
 *               The lower bound on alpha_min keeps the FP32 gain positive.
 *               eta_unsat = 0 selects the default 1.10 used in the paper's experiments.
 *   max_iter:   message-passing rounds, 0 <= max_iter <= 100000 (l_max of Algorithm 1).
 *   flags:      SAGMS_FLAG_* bits.
 * Fields a mode does not use are ignored.
 */
typedef struct {
    int32_t mode;
    float alpha;
    float alpha_min;
    float alpha_max;
    float eta_unsat;
    int32_t max_iter;
    uint32_t flags;
} sagms_params;

/*
 * Load a parity-check matrix (Tanner graph sets M(i), N(j) of Sec. II) onto the current
 * CUDA device.  row_ptr[m+1] and col_idx[nnz] are host arrays in CSR form, columns in any
 * order within a row: the library fixes the edge order (sagms_column_slots), which decides
 * only the order in which a qubit's incoming messages are summed in Eq. 2, i.e. rounding.
 * Requires 1 <= m <= SAGMS_MAX_M, n >= 1, check degrees <= SAGMS_MAX_DC and qubit
 * degrees <= SAGMS_MAX_DV.  On success *out owns device memory until sagms_free_code.
 * Errors: ERR_ARG, ERR_CSR, ERR_DEGREE, ERR_SIZE, ERR_OOM, ERR_CUDA.
 */
int sagms_load_code(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr,
                    const int32_t* col_idx, sagms_code** out);

/* Release a code handle (device memory freed synchronously).  NULL is ignored. */
void sagms_free_code(sagms_code* code);

/* Shape of a loaded code: any output pointer may be NULL. */
int sagms_code_info(const sagms_code* code, int32_t* m, int32_t* n, int32_t* dc_max, int32_t* dv_max);

/* Kernels that can decode a loaded code, in the numbering of a launch plan (sagms_autotune):
 * bit k of *mask set when kernel k has a layout for the code (bit 1, one shot per CTA,
 * always; 2 two-slot; 3 two-group; 4 two-group with column-indexed messages).  Bit 5 (not a
 * plan number): BP has a column-indexed shape of its own for the code (two checks per thread,
 * 129 to 512 or 1025 to 2048 qubits), which BP with per-shot priors takes by default and under plan 4.
 * Parameters can still rule a kernel out: per-qubit priors, no two-group kernel; BP, the
 * one-shot-per-CTA kernel or, with per-shot priors, the column-indexed one.  Host only.
 * Errors: ERR_ARG. */
int sagms_code_kernels(const sagms_code* code, uint32_t* mask);

/*
 * Edge order of the column-indexed kernels (the Sec. II Tanner graph laid out so that a check's
 * edge in slot j keeps its message at row j mod D of its qubit's column).  For every edge e
 * (CSR order) slots[e] in [0, 2D) such that slots are distinct within each check and
 * slots[e] mod D are distinct among each qubit's edges.  The CSR order itself when it has this
 * property (e.g. generalized-bicycle rows listed by polynomial term), else a proper D-edge-
 * colouring of the graph of qubits and check halves (Koenig's theorem: it exists whenever every
 * qubit degree is <= D and every check degree <= 2D), preferring colours that keep cyclic-shift
 * structure.  sagms_load_code uses it with D = the message rows of the kernel shape it picks.
 *   slots  [nnz] host, out (may be NULL when nnz = 0: a code without edges has the empty
 *          assignment).
 * Host only (no CUDA call).  Errors: ERR_ARG (NULL pointers, D outside [1, 32]), ERR_CSR,
 * ERR_DEGREE (a qubit degree above D or a check degree above 2D).
 */
int sagms_column_slots(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr,
                       const int32_t* col_idx, int32_t D, int32_t* slots);

/*
 * Layers of the layered schedule (SAGMS_FLAG_LAYERED): layer[i] for every check i, the
 * smallest layer number used by no check k < i that shares a qubit with check i (first-fit
 * in index order), so the checks of one layer share no qubit.  *num_layers (may be NULL)
 * receives the layer count.
 *   layer  [m] host, out.
 * Host only (no CUDA call).  Errors: ERR_ARG (NULL pointers), ERR_CSR.
 */
int sagms_check_layers(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr,
                       const int32_t* col_idx, int32_t* layer, int32_t* num_layers);

/*
 * The BP rule's phi(x) = -ln tanh(x/2) (Eq. 3) as the decoder evaluates it, for tests of
 * its accuracy: d_y[i] = phi(d_x[i]) for 0 <= d_x[i] <= +inf.  form 0: the decoder's
 * evaluation (two series, one expf or logf each); form 1: the library composition
 * log1pf(2 / expm1f(x)), the reference it is checked against.
 *   d_x, d_y  [n] device.
 * Asynchronous on `stream`.  Errors: ERR_ARG (NULL pointers, n < 0, unknown form), ERR_CUDA.
 */
int sagms_phi(const float* d_x, float* d_y, int64_t n, int32_t form, void* stream);

/* Validate a parameter block without decoding.  Returns SAGMS_OK or SAGMS_ERR_PARAM /
 * SAGMS_ERR_ARG.  Runs on the host only (no CUDA call). */
int sagms_check_params(const sagms_params* params);

/*
 * Decode `shots` syndromes (Algorithm 1, flooding schedule, per-shot early stop).
 *   d_syn   [shots][ceil(m/32)] device, packed input syndromes s.
 *   d_L0    device: [shots] per-shot channel prior L0 = ln((1-q)/q), or [n] per-qubit
 *           priors with SAGMS_FLAG_L0_PER_QUBIT.  A non-finite per-shot prior marks that
 *           shot invalid (err = 0, conv = 0, iters = -1).
 *   d_err   [shots][ceil(n/32)] device, out: packed hard decision e_hat (bit j = 1 iff the
 *           posterior L0_j + sum_{i in N(j)} L_{i->j} is negative).
 *   d_conv  [shots] device, out: 1 if the residual syndrome s XOR H e_hat is zero on return.
 *   d_iters [shots] device, out: message-passing rounds completed when the residual first
 *           became zero (0 for a zero syndrome); max_iter when it never did.
 *   stream  cudaStream_t to launch on (NULL = legacy default stream).
 * The caller owns every buffer; d_syn, d_L0, d_err and d_iters must be 4-byte aligned
 * (ERR_ARG otherwise, before anything is launched).  The library cannot see buffer sizes:
 * each must hold the elements stated above.
 * Asynchronous: results are valid once `stream` has reached this point.  shots == 0 is
 * a no-op.  Errors: ERR_ARG, ERR_PARAM, ERR_SIZE, ERR_OOM, ERR_CUDA.
 */
int sagms_decode(const sagms_code* code, const sagms_params* params, int64_t shots,
                 const uint32_t* d_syn, const float* d_L0, uint32_t* d_err, uint8_t* d_conv,
                 int32_t* d_iters, void* stream);

/*
 * sagms_decode plus a posterior trace for parity checking: d_trace is device memory of
 * [shots][max_iter+1][n] floats; row l receives the posteriors P_j evaluated at the l-th
 * check of Algorithm 1 (l = 0: the prior), in the units the decoder runs in (L0-normalised
 * for the MS family with per-shot priors, LLR units otherwise).  Rows after the shot's
 * last check are left unwritten.
 */
int sagms_decode_trace(const sagms_code* code, const sagms_params* params, int64_t shots,
                       const uint32_t* d_syn, const float* d_L0, uint32_t* d_err, uint8_t* d_conv,
                       int32_t* d_iters, float* d_trace, void* stream);

/*
 * End-to-end decode from HOST buffers: copies syndromes and priors to the device in
 * chunks, decodes, and copies the results back, overlapping the copies of one chunk with
 * the decoding of another on library-owned streams.  Host arrays have the layouts of
 * sagms_decode (h_L0: [shots], or [n] with SAGMS_FLAG_L0_PER_QUBIT); page-locked host
 * memory gives the fastest copies.  Synchronous: returns after all results are in host
 * memory.  Device buffers are allocated from the stream-ordered pool and released before
 * returning.  Errors: as sagms_decode.
 */
int sagms_decode_host(const sagms_code* code, const sagms_params* params, int64_t shots,
                      const uint32_t* h_syn, const float* h_L0, uint32_t* h_err, uint8_t* h_conv,
                      int32_t* h_iters);

/*
 * sagms_decode without any device allocation.  (The paper has no counterpart: this is a
 * deployment variant of sagms_decode.)
 *
 * For callers that cannot allocate device memory while decoding: latency-critical serving
 * threads (cudaMalloc, and cudaMallocAsync when its pool grows, can synchronise or stall
 * the device), processes confined to a device-memory budget fixed at start-up, and host
 * frameworks that own every allocation.  Arguments, layouts and results are those of
 * sagms_decode; results are identical.  The only scratch -- the shot counters the
 * continuous-batching kernels claim shots from -- is a fixed array of SAGMS_NOALLOC_COUNTERS ints in
 * the library's device memory, one counter per launch of up to (2^31 - 1) / W shots
 * (W = max(ceil(m/32), ceil(n/32)) words per pattern; 33.5 million shots at n = 2046), so
 * at most SAGMS_NOALLOC_COUNTERS times that per call; larger batches get SAGMS_ERR_SIZE.
 * Every GPU that loads the library keeps the array until the process exits.
 *   - The first call on a device looks the array's device address up (with that device
 *     current); make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents.  Each call zeroes the
 *     counters it uses on `stream` before launching, so calls that overlap on the GPU (other
 *     streams, other host threads) race: serialise them.
 *   - The call itself allocates nothing: no cudaMalloc / cudaMallocAsync / cudaFree.
 * Errors: as sagms_decode, plus SAGMS_ERR_SIZE for batches beyond the fixed scratch.
 */
#define SAGMS_NOALLOC_COUNTERS 64
int sagms_decode_noalloc(const sagms_code* code, const sagms_params* params, int64_t shots,
                         const uint32_t* d_syn, const float* d_L0, uint32_t* d_err, uint8_t* d_conv,
                         int32_t* d_iters, void* stream);

/*
 * One decode of a batched, mixed-code launch: a code, its parameters and caller-owned
 * device buffers with the layouts of sagms_decode.
 */
typedef struct {
    const sagms_code* code;
    sagms_params params;
    int64_t shots;
    const uint32_t* d_syn;
    const float* d_L0;
    uint32_t* d_err;
    uint8_t* d_conv;
    int32_t* d_iters;
} sagms_job;

/*
 * Decode several batches of possibly different codes (different n and check degrees) in
 * one call: each job runs the decoder of Algorithm 1 exactly as sagms_decode would, on its
 * own library stream forked from `stream` and joined back into it, so the jobs overlap on
 * the GPU and the whole call can be captured into one CUDA graph.  Asynchronous on
 * `stream`.  Errors: as sagms_decode for any job.
 */
int sagms_decode_multi(const sagms_job* jobs, int32_t njobs, void* stream);

/* A captured, instantiated CUDA graph of one sagms_decode_multi call over fixed buffers. */
typedef struct sagms_graph sagms_graph;
int sagms_graph_create(const sagms_job* jobs, int32_t njobs, sagms_graph** out);
int sagms_graph_launch(sagms_graph* graph, void* stream);   /* asynchronous on `stream` */
void sagms_graph_destroy(sagms_graph* graph);

/*
 * Launch-plan autotuning (not part of the method: it picks how the decoder is launched).
 * Decodes the caller's sample batch (buffers as in sagms_decode; the outputs are
 * overwritten) under each candidate plan -- kernel family (two-group or two-slot continuous
 * batching, or one shot per CTA), CTAs per SM, shots per claimed chunk -- times them with
 * CUDA events on `stream` (synchronising it), stores the fastest in the code handle for
 * later decodes, and returns it in *plan with its rate in *shots_per_s.
 * A plan packs: bits 0-2 the kernel (0 automatic, 1 one shot per CTA, 2 two-slot,
 * 3 two-group, 4 two-group with column-indexed messages), bits 8-15 CTAs per SM (0:
 * occupancy limit), bits 16-19 log2 of the shots per claimed chunk (0: automatic); other
 * bits must be zero and the kernel at most 4.  A kernel the code or the parameters cannot
 * use falls back to the next one in the order column-indexed two-group, two-group,
 * two-slot, one shot per CTA.
 * Results of a decode do not depend on the plan.  With the environment variable
 * SAGMS_AUTOTUNE_CACHE naming a file, the plan is also appended there and sagms_load_code
 * of the same matrix starts from it.
 */
int sagms_autotune(const sagms_code* code, const sagms_params* params, int64_t shots,
                   const uint32_t* d_syn, const float* d_L0, uint32_t* d_err, uint8_t* d_conv,
                   int32_t* d_iters, int32_t* plan, float* shots_per_s, void* stream);
int sagms_set_plan(sagms_code* code, int32_t plan);   /* 0 restores the defaults */

/*
 * Largest number of shots one kernel launch of a continuous-batching decode of `code` takes
 * (not part of the method).  A batch is always split into launches of at most
 * (2^31 - 1) / W shots (W = max(ceil(m/32), ceil(n/32)) words per pattern, the kernels'
 * 32-bit shot indexing); a positive `shots` lowers that bound for later decodes of this
 * code, 0 restores it.  Smaller launches bound how long one launch holds the GPU; results do
 * not depend on the split.  sagms_decode_noalloc uses one fixed counter per launch, so its
 * size limit (SAGMS_NOALLOC_COUNTERS launches) follows this bound.
 * Errors: SAGMS_ERR_ARG for a NULL code or shots < 0.
 */
int sagms_set_launch_limit(sagms_code* code, int64_t shots);

/*
 * Serving loop (continuous batching; not part of the method).  A server accepts decode
 * requests -- a registered code, a batch of syndromes and priors in host memory, host output
 * buffers -- at any time from any host thread and runs them on the current device:
 *   - Admission is in arrival order and gated by free device memory: every request's device
 *     buffers come from one arena of `mem_budget` bytes allocated at creation (no request
 *     allocates), and at most `max_inflight` requests are on the GPU at once.
 *   - SAGMS_SERVE_CONTINUOUS: admitted requests run concurrently, each on its own stream
 *     (copy in, decode, copy out); each decode's grid is capped at one CTA per
 *     `shots_per_cta` shots so CTAs of newer requests take SMs as older CTAs retire, and
 *     inside a CTA the decoder refills its shot slots as shots converge.
 *   - SAGMS_SERVE_PLAIN: the baseline -- one request at a time on one stream, full grid.
 * Results are those of sagms_decode for the same code, parameters and inputs.
 * Host buffers must stay valid until the request finishes (page-locked memory copies
 * fastest).  A registered code handle must stay loaded until the server is destroyed.
 * A cancelled request leaves the admission queue at once and may be released right away.
 * Errors: ERR_ARG, ERR_SIZE (request larger than the budget), ERR_BUSY (server
 * stopping, or cancel of a running request), ERR_TIMEOUT (poll), ERR_CANCELLED.
 */
enum { SAGMS_SERVE_CONTINUOUS = 0, SAGMS_SERVE_PLAIN = 1 };
typedef struct sagms_server sagms_server;
int sagms_server_create(size_t mem_budget, int32_t max_inflight, int32_t mode, int32_t shots_per_cta,
                        sagms_server** out);
int sagms_server_add_code(sagms_server* server, const sagms_code* code, const sagms_params* params,
                          int32_t* code_id);
int sagms_server_submit(sagms_server* server, int32_t code_id, int64_t shots, const uint32_t* h_syn,
                        const float* h_L0, uint32_t* h_err, uint8_t* h_conv, int32_t* h_iters,
                        uint64_t* ticket);
/* Wait up to timeout_us (0: just check) for a request; SAGMS_OK once its results are in the
 * host buffers, ERR_TIMEOUT while it is still queued or running. */
int sagms_server_poll(sagms_server* server, uint64_t ticket, int64_t timeout_us);
int sagms_server_cancel(sagms_server* server, uint64_t ticket);   /* queued requests only */
/* Steady-clock nanoseconds at submit and at completion (0 while unfinished). */
int sagms_server_times(sagms_server* server, uint64_t ticket, int64_t* submit_ns, int64_t* done_ns);
int sagms_server_release(sagms_server* server, uint64_t ticket);  /* forget a finished request */
/* Cancels queued requests, waits for running ones, frees the arena. */
int sagms_server_destroy(sagms_server* server);
/* Load generator for measurements: submits request i (arguments as sagms_server_submit,
 * one array entry per request) once arrival_ns[i] nanoseconds have passed since the call
 * began, spinning on the host clock; returns after the last submission with the tickets. */
int sagms_server_replay(sagms_server* server, int32_t n, const int32_t* code_ids, const int64_t* shots,
                        const int64_t* arrival_ns, const uint32_t* const* h_syn, const float* const* h_L0,
                        uint32_t* const* h_err, uint8_t* const* h_conv, int32_t* const* h_iters,
                        uint64_t* tickets);

/* Eq. 9: alpha*(L0, d_c) = 2 atanh(tanh(L0/2)^(d_c - 1)) / L0, the SMS scale matching one
 * BP CN update under uniform inputs (Remark 1).  Returns NaN for L0 <= 0 or d_c < 2. */
double sagms_alpha_star(double L0, int32_t dc);

/*
 * ---- Fused Monte Carlo frame-error estimation (not part of the decoder itself) ----
 *
 * The simulation protocol of Sec. V (setup): for one noise level, draw frames (iid Z flips
 * of each qubit with probability q, the Z part of the memoryless channel of Sec. II), form
 * their syndromes s = H e, decode them with Algorithm 1, and count frame failures until a
 * target number of failures or a maximum number of frames.  Sampling, syndrome formation,
 * decoding and the logical check all run on the GPU; only the counters return to the host.
 *
 * A frame fails when the decoder stops without a zero residual syndrome (the failure exit of
 * Algorithm 1) or when it converges but e XOR e_hat is a nontrivial logical operator (not in
 * the row space of H_Z).  Both kinds are counted separately.
 */
typedef struct {
    int64_t shots;          /* frames decoded */
    int64_t failures;       /* not_converged + logical */
    int64_t not_converged;  /* Algorithm 1 returned its failure exit */
    int64_t logical;        /* converged, but e XOR e_hat is a nontrivial logical operator */
    int64_t iters_sum;      /* sum of the decoder's iteration counts */
} sagms_mc_counts;

/*
 * X-type logical operators of a CSS code: a basis of ker(H_Z) modulo the row space of H_X,
 * k = n - rank(H_X) - rank(H_Z) vectors.  H_X is the decoder's matrix (mx x n), H_Z the
 * other stabilizer matrix (mz x n), both CSR over GF(2).  A Z-type residual r with
 * H_X r = 0 is a stabilizer exactly when x . r = 0 (mod 2) for every returned x.  Host-only
 * (no GPU needed); writes min(k, max_k) packed vectors [k][ceil(n/32)] to `logicals` (may
 * be NULL with max_k = 0 to query k) and k to *k.  Errors: SAGMS_ERR_ARG, SAGMS_ERR_CSR for
 * malformed matrices, SAGMS_ERR_PARAM when H_X H_Z^T != 0 (not a CSS pair).
 */
int sagms_x_logicals(int32_t n, int32_t mx, const int32_t* hx_row_ptr, const int32_t* hx_col_idx,
                     int32_t mz, const int32_t* hz_row_ptr, const int32_t* hz_col_idx, int32_t max_k,
                     uint32_t* logicals, int32_t* k);

/* Attach k >= 0 logical operators (host array [k][ceil(n/32)], copied) to a code for the
 * logical check; k = 0 counts only decoder failures.  Replaces earlier ones. */
int sagms_mc_set_logicals(sagms_code* code, int32_t k, const uint32_t* logicals);

/*
 * Draw frames shot0 .. shot0 + shots - 1 of the generator keyed by `seed`: iid flips with
 * probability q in [0, 1), from Philox4x32-10 (Salmon et al., SC'11) with counter
 * (draw / 4, shot low word, shot high word, 0x53414721) and key (seed low, seed high),
 * each uniform u32 draw giving a run of unflipped qubits by geometric-gap lookup in
 * T[g] = floor((1 - q)^g 2^32) (powers by repeated IEEE double multiplication; T[0] =
 * 2^32 - 1; the run is the largest g <= n with u < T[g]).  This is, bit for bit, the
 * generator the tests use to build inputs.  Writes d_err [shots][ceil(n/32)],
 * d_syn [shots][ceil(m/32)] = H e, and d_L0 [shots] = L0 (the decoder's prior for the
 * level; any of the three may be NULL; those given must be 4-byte aligned, else ERR_ARG
 * before anything is launched).  Asynchronous on `stream`.
 */
int sagms_mc_sample(const sagms_code* code, uint64_t seed, double q, float L0, int64_t shot0, int64_t shots,
                    uint32_t* d_err, uint32_t* d_syn, float* d_L0, void* stream);

/*
 * Logical check of decoded frames against their true errors (device arrays as produced by
 * sagms_mc_sample and sagms_decode): per frame a flag (0 success, 1 not converged,
 * 2 converged to a nontrivial logical) in d_fail (may be NULL), and the counts added to
 * *d_counts (device memory; shots included).  Needs attached logicals.  d_err, d_err_hat
 * and d_iters must be 4-byte aligned and d_counts 8-byte aligned (64-bit atomics), else
 * ERR_ARG before anything is launched.  Asynchronous.
 */
int sagms_mc_check(const sagms_code* code, int64_t shots, const uint32_t* d_err, const uint32_t* d_err_hat,
                   const uint8_t* d_conv, const int32_t* d_iters, uint8_t* d_fail, sagms_mc_counts* d_counts,
                   void* stream);

/*
 * The protocol for one noise level: batches of `batch` frames through sample -> decode ->
 * check until counts->failures >= target_failures or counts->shots >= max_shots.  counts
 * is in/out (host): frames already counted are skipped, so the next frame index is
 * counts->shots and repeated calls continue the same sequence.  The stop is checked between
 * batches, so the last batch can overshoot the failure target.  Synchronous; device
 * buffers come from the stream-ordered pool on a library stream and are released before
 * returning.  Needs attached logicals.
 */
int sagms_mc_run(const sagms_code* code, const sagms_params* params, uint64_t seed, double q, float L0,
                 int64_t target_failures, int64_t max_shots, int64_t batch, sagms_mc_counts* counts);

/* Message of the last failure on the calling thread ("" if none). */
/*
 * Quaternary (GF(4)) decoding (Sec. II; Fig. 2b, Fig. 3 experiments): BP4 and the Min-Sum family
 * on a stabilizer matrix H in GF(4)^{m x n} whose entries are Paulis, with scalar messages
 * (the scalarisation the paper takes from its ref. [Lai_2021]).
 *   - Each qubit holds per-Pauli LLRs Lambda(W) = ln P(I)/P(W), W in {X, Z, Y}, starting at the
 *     prior L0 = ln((1 - eps0) / (eps0/3)); a CN message counts toward Lambda(W) exactly when W
 *     anticommutes with the edge's entry (Eq. 2 read per Pauli).
 *   - The VN->CN message of an edge with entry T is the LLR that the qubit's error commutes with
 *     T: ln(1 + e^{-Lambda'(T)}) - ln(e^{-Lambda'(T')} + e^{-Lambda'(T'')}) over the extrinsic
 *     Lambda' (T', T'' the Paulis anticommuting with T).
 *   - The CN update is the binary rule of Eq. 3 (BP4) or Eqs. 4 / 8 (MS, SMS, SAGMS, gains of
 *     Eqs. 6-7 from the residual of Eq. 1 over GF(4)); decision (Algorithm 1): the argmin of
 *     (0, Lambda(X), Lambda(Z), Lambda(Y)), ties to I, X, Z, Y.  LLR units; clips as sagms_decode.
 *
 * sagms_gf4_load_code: H in CSR (host arrays, copied): row_ptr[m+1], col_idx[nnz], pauli[nnz]
 * with 1 = X, 2 = Z, 3 = Y (the symplectic bits x | z << 1 of Sec. II's map phi_s).
 * 1 <= m <= 512 (one thread per check, 512 per CTA), n <= 16382, check and qubit degree <= 16, no
 * duplicate column in a row.
 * Errors: SAGMS_ERR_ARG, SAGMS_ERR_CSR (bad CSR or Pauli), SAGMS_ERR_DEGREE, SAGMS_ERR_CUDA.
 *
 * sagms_gf4_decode: d_syn [shots][ceil(m/32)] u32 packed syndrome bits s_i = <E, H_i> (trace
 * inner product); d_L0 [shots] f32 one prior LLR per shot (the same for X, Z, Y); outputs
 * d_err [shots][2][ceil(n/32)] u32 (the x bits, then the z bits of e_hat: X = x, Z = z, Y = both),
 * d_conv [shots] u8, d_iters [shots] i32 as sagms_decode.  Parameters as sagms_decode; flags:
 * SAGMS_FLAG_NO_EARLY_STOP and SAGMS_FLAG_GENERIC_KERNEL (below) only.  Device buffers caller-owned, 4-byte aligned; asynchronous on
 * `stream`.  sagms_gf4_decode_trace also writes d_trace [shots][max_iter+1][n][3] f32: Lambda(X),
 * Lambda(Z), Lambda(Y) of every qubit at every checked round.
 * Errors: as sagms_decode, plus SAGMS_ERR_PARAM for other flags and SAGMS_ERR_SIZE when the code's
 * state does not fit a CTA's shared memory.
 *
 * Kernels: a CSS matrix (every row all X or all Z, as the paper's stack of H_X over H_Z) whose
 * rows of each type have a column-indexed slot assignment (sagms_column_slots with D = the
 * largest per-type qubit degree rounded up to a compiled shape: 3, 4, 5, 6 or 8 message rows)
 * is decoded by the column-indexed CSS kernel when its state fits a CTA's shared memory; any
 * other matrix, or SAGMS_FLAG_GENERIC_KERNEL in params->flags, by the generic kernel.  The two
 * run the same rounds and arithmetic per check and qubit and differ only in the order of each
 * qubit's message sums.  sagms_gf4_layout returns 1 when a loaded code takes the CSS kernel,
 * 0 when it takes the generic one, SAGMS_ERR_ARG for a NULL code (no paper counterpart: a
 * property of this library's kernels).
 */
typedef struct sagms_gf4_code sagms_gf4_code;
int sagms_gf4_load_code(int32_t m, int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                        const uint8_t* pauli, sagms_gf4_code** out);
void sagms_gf4_free_code(sagms_gf4_code* code);
int sagms_gf4_layout(const sagms_gf4_code* code);
int sagms_gf4_decode(const sagms_gf4_code* code, const sagms_params* params, int64_t shots, const uint32_t* d_syn,
                     const float* d_L0, uint32_t* d_err, uint8_t* d_conv, int32_t* d_iters, void* stream);
int sagms_gf4_decode_trace(const sagms_gf4_code* code, const sagms_params* params, int64_t shots,
                           const uint32_t* d_syn, const float* d_L0, uint32_t* d_err, uint8_t* d_conv,
                           int32_t* d_iters, float* d_trace, void* stream);

const char* sagms_last_error_string(void);

/* Library version and build constants (clip levels, limits), human-readable. */
const char* sagms_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SAGMS_H */
