/*
 * smnn.h -- C ABI of libsmnn, the batched linear-time solve of the reformulated
 * Mechanistic Neural Network layer (Scalable Mechanistic Neural Networks,
 * Chen et al., ICLR 2025), with hand-written CUDA kernels for sm_103a.
 *
 * The problem (Sec. 3.1).  A *system* is one (sequence b, dimension dd) pair with
 * V = Q = 1: T steps, R+1 unknowns y_{t,0..R} per step (the value and its first R
 * derivatives), and the weighted least-squares problem
 *     y = argmin || W^{1/2} (A y - b) ||^2,   i.e.  M y = beta,  M = A^T W A   (Eq. 9)
 * built from one governing row per step (Eq. 4: sum_r c_{t,r} y_{t,r} = d_t), the
 * initial-value rows (Eq. 5: y_{t,r} = u_{t,r}, t <= T_init, r <= R_init) and the
 * forward/backward Taylor smoothness rows between adjacent steps (Eq. 6-7, weight
 * (w_smooth s_t^r)^2).  With the unknowns ordered by step (Sec. 3.2, Eq. m_partition)
 * M is symmetric positive definite and block tridiagonal with (R+1)x(R+1) blocks:
 * M_t on the diagonal and N_t at block (t+1, t); M_t, N_t and beta_t have the closed
 * forms of App. A.2.  The library never forms A.
 *
 * Layouts (all arrays row-major, contiguous, caller-owned DEVICE memory unless stated):
 *   uniform batch (desc.seq_T == NULL), S = B*D systems, system i = b*D + dd:
 *     c  [B][D][T][R+1]   coefficients c_{t,r} of Eq. 4
 *     d  [B][D][T]        right-hand sides d_t of Eq. 4
 *     s  [B][T]           step sizes s_t (Eq. 6-7), shared by the D systems of a
 *                         sequence; s[b][T-1] is unused
 *     u  [B][D][T_init][R_init+1]   initial values of Eq. 5
 *     y  [B][D][T][R+1]   solution (same layout as c)
 *   ragged batch (desc.seq_T = per-sequence step counts T_b): the D systems of
 *     sequence b are stored one after another, system i = b*D + dd starting at
 *     step D*(T_0+...+T_{b-1}) + dd*T_b of c, d, y (c and y hold R+1 values per
 *     step); s holds T_0+...+T_{B-1} entries, sequence b starting at T_0+...+T_{b-1};
 *     u is [S][T_init][R_init+1].
 *   Element type: float for SMNN_F32_REFINED and SMNN_F32, double for SMNN_F64.
 *
 * Streams: every compute call is asynchronous and ordered on the given stream
 * (a cudaStream_t passed as void*; NULL = legacy default stream); it allocates
 * nothing and does not synchronise.  Host return codes report argument, workspace
 * and launch errors only.  Numerical failures go to the device array info[S]
 * (int32): 0 ok; k > 0: a non-positive pivot was met at (1-based) step k of that
 * system, and its outputs are NaN (steps eliminated first are reported first: a failure
 * inside a chunk is reported before the separators it poisons); -1: the refinement stop test
 * (desc.refine_tol > 0) was not met after the last sweep.
 */
#ifndef SMNN_H_
#define SMNN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest derivative order the kernels are compiled for (R+1 <= 4 unknowns/step). */
#define SMNN_MAX_R 3
/* Largest block n_b = V(R+1) and equation count Q of a coupled step (smnn_desc.V, .Q). */
#define SMNN_MAX_NB 9
#define SMNN_MAX_Q 3

typedef enum {
  SMNN_OK = 0,
  SMNN_ERR_INVALID_ARG = 1,   /* a pointer, size or parameter is out of range      */
  SMNN_ERR_WORKSPACE = 2,     /* workspace/factor buffer missing or misaligned     */
  SMNN_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed       */
  SMNN_ERR_UNSUPPORTED = 4,   /* valid request the library does not implement     */
  SMNN_ERR_TOO_LARGE = 5      /* exceeds the static scratch of smnn_factor_solve_noalloc */
} smnn_status;

typedef enum {
  /* FP32 factorisation and substitution, accuracy won back by iterative refinement whose
   * residual r = beta - M y is evaluated in FP64 from the FP32 inputs; the refined
   * solutions are accumulated as float-float pairs (float arrays). */
  SMNN_F32_REFINED = 0,
  SMNN_F32 = 1,   /* FP32 factorisation and substitution only (float arrays)         */
  SMNN_F64 = 2,   /* plain FP64 block Cholesky of the same method (double arrays)    */
  /* As SMNN_F32_REFINED, but the residual and the gradient formulas are evaluated in
   * float-float arithmetic (pairs of FP32 numbers combined with error-free
   * transformations, ~48-bit significand) on the FP32 pipe instead of in FP64. */
  SMNN_F32_REFINED_DF = 3
} smnn_precision;

typedef enum {
  SMNN_ALGO_AUTO = 0,  /* chunked reduction, one launch per level and direction up   */
                       /* to the first level whose systems each fit a CTA (<= 128    */
                       /* chunks), one launch for that level and all above it        */
  SMNN_ALGO_SEQ = 1,   /* one sequential block-Cholesky sweep per system (Alg. 3, 4), */
                       /* elimination and substitution in one launch                 */
  SMNN_ALGO_CR = 2,    /* chunked block cyclic reduction, parallel over T, one       */
                       /* launch per level and direction                             */
  SMNN_ALGO_CR_FUSED = 3 /* chunked reduction in one launch per solve pass: a CTA runs */
                       /* every level of its systems; plan creation returns          */
                       /* SMNN_ERR_UNSUPPORTED when a system has more than 128       */
                       /* level-0 chunks                                             */
} smnn_algo;

typedef struct smnn_desc {
  int32_t R;              /* highest derivative order, 1..SMNN_MAX_R                */
  int32_t R_init;         /* initial values for orders 0..R_init, 0 <= R_init <= R  */
  int32_t T_init;         /* initial values for steps 1..T_init, 1 <= T_init <= T_b */
  int32_t precision;      /* smnn_precision                                         */
  int32_t algo;           /* smnn_algo                                              */
  int32_t max_refine;     /* forward refinement sweeps (refined modes), 0..16       */
  int32_t chunk;          /* level-0 chunk length of the chunked reduction, 0 = auto */
  int32_t adjoint_refine; /* refinement sweeps of the adjoint solve, 0..16; when > 0 */
                          /* the backward also refines y once before the gradients  */
  double w_gov;           /* importance weights of Eq. 9 (unsquared; W holds their  */
  double w_init;          /*   squares, App. A.1), >= 0                             */
  double w_smooth;
  double refine_tol;      /* > 0: per-system stop test of the refinement: a system   */
                          /* stops once its estimated error ||dy_k||^2/||dy_{k-1}|| */
                          /* is <= refine_tol ||y|| (the remaining sweeps skip it);  */
                          /* still above after the last sweep: info = -1            */
  int64_t num_seq;        /* B >= 1                                                 */
  int64_t dims_per_seq;   /* D >= 1                                                 */
  int64_t T;              /* steps per sequence (uniform batch; ignored if seq_T)   */
  const int64_t* seq_T;   /* HOST pointer to B step counts (ragged), or NULL; read  */
                          /* only during smnn_plan_create                           */
  int32_t V;              /* variables per step (Sec. 3.1; 0 means 1): a step has   */
                          /* n_b = V(R+1) <= SMNN_MAX_NB unknowns, variable-major   */
  int32_t Q;              /* governing equations per step (0 means 1), 1..MAX_Q;   */
                          /* with V and Q the per-step layouts become              */
                          /* c [..][Q][V(R+1)], d [..][Q], u [..][T_init][V][R_init+1], */
                          /* y [..][V(R+1)] (gradients likewise).  Built shapes:   */
                          /* V = Q = 1 with R = 1..3; V = 2, R = 1, Q = 1 or 2;    */
                          /* V = 3, R = 1, Q = 3; V = 2, R = 2, Q = 2; V = 3, R = 2, */
                          /* Q = 3 (n_b = 9).  Other valid                         */
                          /* shapes return SMNN_ERR_UNSUPPORTED at plan creation.   */
  int32_t per_level_launches; /* 0 (default): refined FP32 solves of AUTO plans with   */
                          /* two levels and at most 32 level-0 chunks per system run  */
                          /* one warp per system, one launch per pass boundary;      */
                          /* nonzero: one launch per level, pass and stop test there */
                          /* too (the same arithmetic; for comparison and testing)   */
} smnn_desc;

typedef struct smnn_plan_s* smnn_plan;

typedef struct smnn_plan_stats {
  int64_t num_systems;    /* S = B*D                                                */
  int64_t total_steps;    /* sum over systems of T_i                                */
  int32_t num_levels;     /* reduction levels of the solve (1 = sequential)         */
  int32_t chunk[8];       /* chunk length per level                                 */
  int32_t kernels_per_solve;
  size_t workspace_bytes; /* as smnn_workspace_size                                 */
  size_t factor_bytes;
} smnn_plan_stats;

/* Validate desc and build a plan: the level structure of the chunked reduction
 * and its small device index tables.  This is the only call that allocates (device
 * memory for the tables).  Returns SMNN_ERR_INVALID_ARG for out-of-range fields,
 * SMNN_ERR_CUDA if the tables cannot be allocated.  The plan is bound to the device
 * current at creation. */
smnn_status smnn_plan_create(const smnn_desc* desc, smnn_plan* plan);

/* Free a plan and its tables (synchronises the device first). NULL is a no-op. */
smnn_status smnn_plan_destroy(smnn_plan plan);

/* Level structure and buffer sizes of a plan (host call, no GPU work). */
smnn_status smnn_plan_get_stats(smnn_plan plan, smnn_plan_stats* stats);

/* Bytes of device workspace the compute calls need (workspace_bytes, 256-byte
 * aligned base required), and the bytes of the optional saved factor (the Cholesky
 * blocks L_t of Sec. 3.2 Eq. 11-12 in the plan's chunked order, with the fill
 * blocks and reduced blocks of the reduction) that smnn_factor_solve can leave for
 * smnn_backward. */
smnn_status smnn_workspace_size(smnn_plan plan, size_t* workspace_bytes, size_t* factor_bytes);

/* App. A.2: materialise M_t (lower triangle packed row by row: M_00, M_10, M_11,
 * M_20, ..., n_b(n_b+1)/2 values), N_t (block (t+1,t), n_b^2 values row-major,
 * zero for the last step of a system) and beta_t (n_b values) for every step, laid
 * out per step like y; n_b = V(R+1) (for V > 1 the smoothness part of M_t and N_t is
 * block diagonal over the variables, the governing part sum_q w_gov^2 c_q c_q^T).  workspace: as for smnn_factor_solve.  Testing and inspection
 * aid; the solver forms these blocks in registers. */
smnn_status smnn_assemble(smnn_plan plan, const void* c, const void* d, const void* s,
                          const void* u, void* M, void* N, void* beta, void* workspace,
                          void* stream);

/* Forward pass (Alg. 1: Decompose, Alg. 3, then Substitute, Alg. 4, in the chunked
 * cyclic-reduction order of the plan), fused with the assembly of App. A.2, plus
 * max_refine refinement sweeps for SMNN_F32_REFINED.  Writes y and info.
 * factor: NULL, or a factor_bytes buffer (256-byte aligned) that receives the factor
 * for smnn_backward.  workspace: workspace_bytes of device scratch (256-byte aligned). */
smnn_status smnn_factor_solve(smnn_plan plan, const void* c, const void* d, const void* s,
                              const void* u, void* y, void* factor, int32_t* info,
                              void* workspace, void* stream);

/* Backward pass (Alg. 2 and Eq. 14): g = M^{-1} dl/dy with the same factor (refined
 * like the forward pass), then the parameter gradients, fused per step as the chain
 * rule through App. A.2's assembly (per governing equation q when Q > 1; per variable
 * v for the initial values and the smoothness rows when V > 1):
 *   gd_t = w_gov^2 c_t.g_t,   gc_t = w_gov^2 [(d_t - c_t.y_t) g_t - (c_t.g_t) y_t],
 *   gu_{t,r} = w_init^2 g_{t,r},
 *   gs_t = -w_smooth^2 d/ds_t sum_r s_t^{2r} (f+_r e+_r + f-_r e-_r), summed over the
 *          D systems of the sequence, with e+ = exp(s_t N) y_t - y_{t+1},
 *          e- = exp(-s_t N) y_{t+1} - y_t (f+- likewise on g, N the nilpotent shift);
 *          gs of the last step of a sequence is 0.
 * y: the forward solution; gy: dl/dy (layout of y).  factor: the buffer filled by
 * smnn_factor_solve with the same inputs, or NULL to recompute the factor into the
 * workspace.  Outputs gc, gd, gs, gu have the layouts of c, d, s, u.
 * gw: NULL, or 3 doubles of device memory (8-byte aligned) that receive the derivatives
 * of the loss with respect to the importance weights of Eq. 9, shared by all systems of
 * the batch (App. A.1: each row's weight is the square of w times a step-size power):
 *   gw[0] = dl/dw_gov    = 2 w_gov sum_t (c_t.g_t)(d_t - c_t.y_t),
 *   gw[1] = dl/dw_init   = 2 w_init sum_{t<T_init, r<=R_init} g_{t,r} (u_{t,r} - y_{t,r}),
 *   gw[2] = dl/dw_smooth = -2 w_smooth sum_t sum_r s_t^{2r} (f+_r e+_r + f-_r e-_r),
 * summed over every system whose info is 0, in a fixed order (deterministic); the terms
 * are formed in the precision of the residual and summed in FP64. */
smnn_status smnn_backward(smnn_plan plan, const void* c, const void* d, const void* s,
                          const void* u, const void* y, const void* factor, const void* gy,
                          void* gc, void* gd, void* gs, void* gu, double* gw, int32_t* info,
                          void* workspace, void* stream);

/* A captured step: smnn_factor_solve on (c, d, s, u) into (y, factor, info) and, when gy
 * is not NULL, smnn_backward on dl/dy = gy into (gc, gd, gs, gu, gw, info_b), recorded once
 * into a CUDA graph on fixed buffers and replayed by smnn_graph_launch as one launch in place
 * of the step's ~40 kernel launches (Sec. 6 names launch overhead as what dominates batches
 * of small systems).  Arguments keep their meaning, layout, alignment and NULL rules from
 * smnn_factor_solve and smnn_backward; the buffers must stay allocated at the same
 * addresses while the graph exists, and new inputs are written into them between launches.
 * The capture runs on a private stream of the plan's device in thread-local capture mode
 * and executes nothing; the plan must outlive the graph.  The profiler does not time graph
 * launches; smnn_launch_count grows by the graph's kernel count at every launch.
 * On failure *graph is NULL and nothing is left allocated. */
typedef struct smnn_graph_s* smnn_graph;
smnn_status smnn_graph_create(smnn_plan plan, const void* c, const void* d, const void* s,
                              const void* u, void* y, void* factor, int32_t* info,
                              const void* gy, void* gc, void* gd, void* gs, void* gu,
                              double* gw, int32_t* info_b, void* workspace, smnn_graph* graph);
/* Replays the step on `stream` (stream-ordered, asynchronous, on the plan's device). */
smnn_status smnn_graph_launch(smnn_graph graph, void* stream);
/* Frees the graph (NULL is a no-op); launches already issued are not affected. */
smnn_status smnn_graph_destroy(smnn_graph graph);

/* Per-kernel timing of this library's own launches, for benchmarks.  While enabled
 * (enable != 0), every kernel launch is bracketed by two CUDA events recorded on the
 * launch's stream; up to 65536 launches are kept, later ones are counted but not timed.
 * smnn_profile_enable creates the events when called with enable != 0 and clears the
 * record; it must not be called during stream capture. */
smnn_status smnn_profile_enable(int enable);

typedef struct smnn_kernel_time {
  char name[48];          /* kernel name (template arguments stripped)             */
  int64_t launches;       /* launches recorded while enabled                        */
  double total_ms;        /* sum of their event-measured durations                  */
} smnn_kernel_time;

/* Synchronise on the recorded events and aggregate them by kernel name into out[0..n),
 * at most max entries; *n receives the number of distinct kernels. */
smnn_status smnn_profile_read(smnn_kernel_time* out, int max, int* n);

/* Forward solve without any device allocation.  The paper has no counterpart: this entry
 * point is for callers that may not allocate device memory at all -- code that runs
 * under an allocator that owns every device byte (a framework's caching pool, an
 * embedding application), code on a path where cudaMalloc's implicit synchronisation or
 * possible failure is not acceptable (latency-critical or real-time loops), and code that
 * cannot keep a plan alive between calls.  It computes what smnn_plan_create followed by
 * smnn_factor_solve (with factor = NULL) computes for the same desc and inputs, but takes
 * no plan and no workspace: the plan's index tables and the workspace are placed in one
 * library-owned static device array of SMNN_NOALLOC_SCRATCH_BYTES (64 MiB) per device,
 * held by every GPU that loads the library until the process exits.
 *   - Requests whose tables plus workspace exceed that size return SMNN_ERR_TOO_LARGE and
 *     launch nothing (smnn_workspace_size of an equivalent plan tells the need).
 *   - The call allocates no device memory (no cudaMalloc, cudaFree or allocating library
 *     routine); it uses host memory for the plan's bookkeeping and copies the index tables
 *     to the device with cudaMemcpyAsync on `stream`.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (once per device, with that device current); make that first
 *     call before any stream capture.
 *   - All calls on a device share the one array, which keeps the previous call's contents;
 *     everything the solve reads is written earlier in the same call (info is cleared by
 *     the call itself).  Calls that overlap on the GPU -- on different streams, or from
 *     different host threads without ordering -- race on the array and give wrong results.
 * Arguments, layouts and info as smnn_factor_solve; desc as smnn_plan_create. */
#define SMNN_NOALLOC_SCRATCH_BYTES (64u << 20)
smnn_status smnn_factor_solve_noalloc(const smnn_desc* desc, const void* c, const void* d,
                                      const void* s, const void* u, void* y, int32_t* info,
                                      void* stream);

/* Arithmetic peak of the current device, for roofline reports (no counterpart in the
 * paper): the rate of fused multiply-adds, FP32 (fp64 = 0) or FP64 (fp64 != 0), measured
 * by chains of dependent FMAs, eight independent chains per thread, at full occupancy
 * (eight CTAs of 256 threads per SM), as the better of two timed launches of ~50 ms after
 * a warm-up launch on `stream`.  Synchronous: returns after the timing with
 * *fma_per_s set (one FMA = 2 flops).  Allocates a few bytes of device memory for the
 * kernel's sink and frees them.  SMNN_ERR_CUDA on any CUDA error. */
smnn_status smnn_fma_rate(int32_t fp64, double* fma_per_s, void* stream);

/* Static string for a status code. */
const char* smnn_status_string(smnn_status status);

/* Number of kernels this library has launched in this process (all devices). */
uint64_t smnn_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SMNN_H_ */
