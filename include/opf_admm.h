/*
 * opf_admm.h -- C ABI of the B300 (sm_103a) solver-free componentwise ADMM
 * for linearized multi-phase optimal power flow in distribution feeders.
 *
 * Method (arxiv 2501.08293):
 *   model       Section II-A, Eqs. (operational), (balance_eqns),
 *               (volt_load_model) VDLM-1..10, (power_flow_eqns), objective
 *               sum of pg; abstract LP of Eq. (LP_model).
 *   decompose   Eq. (OurModel): equality rows stay in the components
 *               (bus, line, load, generator), every bound moves to the
 *               global vector x.
 *   precompute  Section IV-B row reduction and Eq. (closed_2):
 *               Abar_s = A_s^T (A_s A_s^T)^{-1} A_s - I,
 *               bbar_s = A_s^T (A_s A_s^T)^{-1} b_s.
 *   iterate     Algorithm 1: global update Eq. (global_sparse), local update
 *               Eq. (closed_2), dual update Eq. (ADMM-3); residuals and
 *               stopping test of Eq. (termination).
 *
 * Conventions
 *   - Every function returns an int32 status (opf_status); nothing throws or
 *     aborts across the ABI.  opf_last_error() gives a message for the last
 *     failing call on the calling thread.
 *   - Input records are read during the call and copied; the caller keeps
 *     ownership of every buffer it passes.
 *   - A problem handle owns its host data, its pinned host buffers and (when
 *     it allocated them itself) its device buffers.  One handle must not be
 *     used by two threads at once; distinct handles are independent.
 *   - "stream" arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).  Device work is enqueued on that stream.
 *   - Per-unit quantities throughout.  Phase sets are bit masks a=1, b=2,
 *     c=4; per-phase arrays are indexed 0..2 = a, b, c and entries of absent
 *     phases are ignored on input and written as NaN on output.
 *   - Bounds may be +-INFINITY (a variable counts as bounded only when both
 *     bounds are finite, which matters for the initial point).
 */
#ifndef OPF_ADMM_H
#define OPF_ADMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OPF_ABI_VERSION 1

/* ------------------------------------------------------------ status codes */
enum {
    OPF_OK = 0,                 /* converged (or finished as asked)              */
    OPF_NOT_CONVERGED = 1,      /* max_iter reached; the iterate is still valid  */
    OPF_ERR_INVALID_ARG = -1,   /* bad pointer, size, index, phase set or value  */
    OPF_ERR_INCONSISTENT = -2,  /* row reduction met 0 = b, b != 0 (Sec. IV-B)   */
    OPF_ERR_NUMERIC = -3,       /* NaN / Inf in the residuals or a singular Gram */
    OPF_ERR_OOM = -4,           /* host or device allocation failed              */
    OPF_ERR_CUDA = -5,          /* a CUDA runtime call failed                    */
    OPF_ERR_TIMEOUT = -6,       /* a bounded device wait gave up                 */
    OPF_ERR_STATE = -7          /* call out of order (e.g. solve before upload)  */
};

/* ----------------------------------------------------------- input records
 * Layouts are fixed (sizes 104, 376, 128, 104 bytes); opf_record_size()
 * returns them so bindings can check their own copies.                      */

/* Bus i: squared voltage magnitude bounds (Eq. operational) and shunt
 * conductance / susceptance g^sh, b^sh (Eq. balance_eqns).                  */
typedef struct opf_bus {
    uint8_t phases;
    uint8_t _pad[7];
    double w_lo[3], w_hi[3];
    double g_sh[3], b_sh[3];
} opf_bus;

/* Line e from bus i (from_bus) to bus j (to_bus), Eq. (power_flow_eqns):
 * r, x are 3x3 row-major over phases a, b, c (only the rows/columns of the
 * line's phases are read -- the M^p, M^q sub-block); g_fr, b_fr = g^s_eij,
 * b^s_eij (from end), g_to, b_to = g^s_eji, b^s_eji (to end); tap = tau_e;
 * flow bounds apply to both p_eij and p_eji (and q).  Lines with
 * in_service == 0 are left out of the model.                                */
typedef struct opf_line {
    int32_t from_bus, to_bus;
    uint8_t phases, in_service;
    uint8_t _pad[6];
    double r[9], x[9];
    double g_fr[3], b_fr[3], g_to[3], b_to[3];
    double tap[3];
    double p_lo[3], p_hi[3], q_lo[3], q_hi[3];
} opf_line;

/* Generator k at bus: bounds on pg, qg (Eq. operational) and the linear cost
 * of pg per phase (the paper's objective is cost = 1).                      */
typedef struct opf_gen {
    int32_t bus;
    uint8_t phases;
    uint8_t _pad[3];
    double pg_lo[3], pg_hi[3], qg_lo[3], qg_hi[3];
    double cost[3];
} opf_gen;

/* Load l at bus, Eq. (volt_load_model): conn 0 = wye (VDLM-5), 1 = delta
 * (VDLM-6..10; three-phase only, else OPF_ERR_INVALID_ARG); a, b, alpha,
 * beta as in VDLM-1/2.                                                      */
typedef struct opf_load {
    int32_t bus;
    uint8_t phases, conn;
    uint8_t _pad[2];
    double a[3], b[3], alpha[3], beta[3];
} opf_load;

/* ------------------------------------------------------------- parameters */
enum { OPF_CRIT_ABS = 0, OPF_CRIT_REL = 1, OPF_CRIT_BOTH = 2, OPF_CRIT_NEVER = 3 };
enum { OPF_FP64 = 0, OPF_FP32 = 1 };
/* Residual form of Eq. (termination).  PAPER (as printed): the sum over
 * components outside the norm, dres = rho sqrt(sum_s ||B_s^T (x_s -
 * x_s_prev)||^2) and eps_dual = eps_rel sqrt(sum_s ||B_s^T lambda_s||^2);
 * since B_s^T only places entries, these equal rho ||x_loc - x_loc_prev||
 * and eps_rel ||lambda|| over the stacked locals.  TEXTBOOK: the sum inside
 * the norm, dres = rho ||sum_s B_s^T (x_s - x_s_prev)|| and eps_dual =
 * eps_rel ||sum_s B_s^T lambda_s|| (per global variable, the copies'
 * changes and duals added up first).  pres and eps_prim are the same in
 * both.  TEXTBOOK runs on the GRAPH and HOSTLOOP engines (AUTO picks GRAPH;
 * PERSISTENT, batches, scenarios and the server answer OPF_ERR_INVALID_ARG). */
enum { OPF_RES_PAPER = 0, OPF_RES_TEXTBOOK = 1 };
enum { OPF_ENGINE_AUTO = 0, OPF_ENGINE_GRAPH = 1, OPF_ENGINE_HOSTLOOP = 2, OPF_ENGINE_PERSISTENT = 3 };

/* Solve parameters.  criterion ABS: pres <= eps_abs_prim and dres <=
 * eps_abs_dual; REL: the paper's relative test of Eq. (termination) with
 * eps_rel; BOTH: both; NEVER: run exactly max_iter iterations.  Residuals
 * and the test are evaluated every check_every iterations (the stop can be
 * up to check_every-1 iterations late).  warm_start 0 restarts from the
 * initial point of Section V-A; 1 continues from the handle's current state
 * (iteration counter included).  engine GRAPH runs the whole loop as one
 * CUDA graph with a device-side while node; HOSTLOOP checks from the host;
 * PERSISTENT runs it as one cooperative kernel whose CTAs own feeder chunks
 * and wait only on neighbouring chunks (every wait bounded in time, see
 * opf_debug_config); AUTO picks PERSISTENT when the chunks fit co-resident
 * on the device, else GRAPH.
 * adaptive_rho 1 enables residual balancing, the acceleration the paper
 * names in Section III-D: at every residual check that does not stop,
 * rho *= rb_tau when pres > rb_mu * dres and rho /= rb_tau when dres >
 * rb_mu * pres (duals are unscaled, so they are kept; the operators do not
 * depend on rho).  The current rho is reported in opf_info.rho.            */
typedef struct opf_params {
    double rho;
    double eps_abs_prim, eps_abs_dual, eps_rel;
    int32_t criterion;
    int32_t max_iter;
    int32_t check_every;
    int32_t precision;
    int32_t residual_form;
    int32_t warm_start;
    int32_t engine;
    int32_t adaptive_rho;
    double rb_mu, rb_tau;
} opf_params;

/* Result of a solve.  iters counts all iterations since the last cold
 * start; first_rel_iter is the first checked iteration at which the paper's
 * relative test held (-1 if never); seconds is host wall time of the call. */
typedef struct opf_info {
    int32_t status;
    int32_t iters;
    int32_t first_rel_iter;
    int32_t rho_changes;     /* residual-balancing updates of rho in this solve */
    double pres, dres, eps_prim, eps_dual;
    double objective;
    double seconds;
    double rho;              /* rho at the end of the solve                     */
} opf_info;

/* Sizes of a built problem. */
typedef struct opf_dims {
    int32_t n_global;        /* n: global variables (Eq. LP_model column count) */
    int32_t n_local;         /* sum_s n_s: stacked local copies                 */
    int32_t n_comp;          /* S                                              */
    int32_t n_rows;          /* sum_s m_s before row reduction                  */
    int32_t n_rows_reduced;  /* sum_s m_s after row reduction                   */
    int32_t max_n;           /* max_s n_s                                      */
    int32_t n_tiles;         /* warp tiles of the local-update kernel           */
    int32_t n_blocks;        /* feeder chunks = CTAs of the local update        */
    int64_t sum_n2;          /* sum_s n_s^2 (dense operator entries)            */
    int64_t device_bytes;    /* bytes opf_problem_upload needs                  */
    int32_t max_chunk_locals;    /* largest chunk: locals                       */
    int32_t max_chunk_halo;      /* largest chunk: globals it copies            */
    int32_t max_chunk_operator;  /* largest chunk: operator elements            */
    int32_t max_chunk_copies;    /* largest chunk: halo copy-list entries       */
} opf_dims;

typedef struct opf_problem opf_problem;

/* ------------------------------------------------------------ entry points */

int32_t opf_abi_version(void);
/* which: 0 bus, 1 line, 2 gen, 3 load, 4 params, 5 info, 6 dims; else 0.   */
size_t opf_record_size(int32_t which);
const char* opf_status_string(int32_t status);
const char* opf_last_error(void);
void opf_params_default(opf_params* p);   /* rho 100, ABS 1e-4, eps_rel 1e-3 */

/* Build the model of Section II-A from the records, split it into fine
 * components (Eq. OurModel), row-reduce each [A_s | b_s] and precompute the
 * closed-form operators of Eq. (closed_2) in FP64 on the host, then pack
 * them for the device.  No device memory is touched.
 * Errors: INVALID_ARG (indices, phases, delta on < 3 phases, lo > hi, NaN),
 * INCONSISTENT (a component's rows have no solution), OOM.                  */
int32_t opf_problem_create(const opf_bus* buses, int32_t n_bus,
                           const opf_line* lines, int32_t n_line,
                           const opf_gen* gens, int32_t n_gen,
                           const opf_load* loads, int32_t n_load,
                           opf_problem** out);

/* Decomposition into components (Eq. OurModel).  FINE: one component per
 * bus, in-service line, load and generator.  PAPER: the decomposition of
 * Section V-A -- one component per node of the feeder graph (a bus with its
 * loads and generators) and one per in-service line, a leaf node (a bus
 * with exactly one in-service line) being combined with that line, so S =
 * nodes + lines - leaves (Table III).  Canonical orders under PAPER:
 * components = non-leaf nodes (bus order), then in-service lines (line
 * order); a node's locals = its bus locals, then each load's pd, qd (pb, qb
 * and w are already there), generators adding none; a line with leaf ends =
 * the line locals, then the from-end node's remaining locals if it is a
 * leaf, then the to-end node's; rows stacked in the same order.
 * opf_get_structure reports a node as kind 0 (bus) and a line component as
 * kind 1, with the bus or line index.                                      */
enum { OPF_DECOMP_FINE = 0, OPF_DECOMP_PAPER = 1 };

/* Layout options for opf_problem_create_ex.  chunks = number of feeder
 * chunks (CTAs of the local update; 0 = automatic: about one per 4096 units
 * of n_s^2 + 4 n_s + 16, at most 296).  Batches give each instance a share
 * of the device so that all of them run co-resident.  decomposition =
 * OPF_DECOMP_FINE (default, 0) or OPF_DECOMP_PAPER.                        */
typedef struct opf_create_options {
    int32_t chunks;
    int32_t decomposition;
    int32_t _reserved[6];
} opf_create_options;

/* opf_problem_create with layout options (NULL = defaults).                */
int32_t opf_problem_create_ex(const opf_bus* buses, int32_t n_bus,
                              const opf_line* lines, int32_t n_line,
                              const opf_gen* gens, int32_t n_gen,
                              const opf_load* loads, int32_t n_load,
                              const opf_create_options* options, opf_problem** out);

int32_t opf_get_dims(const opf_problem* p, opf_dims* dims);

/* Tuning table of the automatic chunking (opf_create_options.chunks = 0;
 * the paper has no counterpart: its CPU runs spread the components evenly
 * over N workers, Section V-A).  A problem of n_bus buses is cut into
 * chunks of about work_per_chunk units of n_s^2 + 4 n_s + 16, at most
 * max_chunks; an entry applies to the GPU whose cudaDeviceProp::name equals
 * `gpu` ("*" matches any) and to n_bus_lo <= n_bus < n_bus_hi.  Without a
 * matching entry: 4096 units, at most 296 chunks.  Entries are process-wide
 * (guarded by a mutex) and replace one with the same gpu and bucket.
 * opf_tuning_load reads the JSON file the project's tuner writes
 * ({"gpu": name, "entries": [{"n_bus_lo", "n_bus_hi", "work_per_chunk",
 * "max_chunks", ...}]}, other keys ignored; *n_entries may be NULL);
 * opf_tuning_lookup reports what a create on the current device would use.
 * Errors: INVALID_ARG (unreadable or malformed file, values out of range:
 * 0 <= lo < hi, 16 <= work_per_chunk <= 2^26, 1 <= max_chunks <= 65536).   */
int32_t opf_tuning_set(const char* gpu, int32_t n_bus_lo, int32_t n_bus_hi, int32_t work_per_chunk,
                       int32_t max_chunks);
int32_t opf_tuning_clear(void);
int32_t opf_tuning_load(const char* path, int32_t* n_entries);
int32_t opf_tuning_lookup(int32_t n_bus, int32_t* work_per_chunk, int32_t* max_chunks);

/* New parameters for in-service lines of an uploaded problem: records[k]
 * replaces line line_idx[k] (impedances r, x; shunts; taps; flow bounds).
 * Ends, phases and the service state must not change (a switch in or out
 * of service is opf_set_line_status), else OPF_ERR_INVALID_ARG before
 * anything changes.  The touched components'
 * operators of Eq. (closed_2) are recomputed on the device in FP64
 * (Cholesky of A_s A_s^T; the rows of a line are of full rank) and written
 * into both precisions; the iterate and duals are kept, so a following
 * solve with warm_start continues from them.  OPF_ERR_STATE before upload.
 * The paper precomputes once per topology; this is the incremental update
 * for parameter changes (tap changers, ratings) at high rate.            */
int32_t opf_update_lines(opf_problem* p, const int32_t* line_idx, const opf_line* records, int32_t count,
                         void* stream);

/* Switch line `line` (index in the input records) in (in_service = 1) or
 * out of service (0): the paper's dynamically changing topology
 * (Section I; the model of Section II-A leaves out lines that are out of
 * service).  The line's flows appear in or leave the global vector and the
 * rows of the components at its ends change, so the model is assembled
 * again from the records the problem was built from (with every earlier
 * opf_update_lines / opf_set_line_status applied) and the operators of
 * Eq. (closed_2) are recomputed for the components whose rows changed only
 * (*n_recomputed, may be NULL, gets their number; every other component
 * keeps its operator).  Same decomposition and chunk option as at create.
 * On an uploaded problem the new layout is uploaded to the problem's
 * device (the handle then allocates its own arena with cudaMallocAsync on
 * `stream`; an arena the caller passed to opf_problem_upload is no longer
 * used once the call returns) and the iterate and duals are carried over
 * on the device for every local copy whose component (kind, element) and
 * global variable (element, phase) exist before and after; new copies start
 * from the initial point of Section V-A.  The next solve with warm_start =
 * 1 continues from there; the iteration counter restarts at 0.  The call
 * synchronizes `stream`.  Batches that include the problem must be created
 * again.  No change when the line already has that state.  Closing a line
 * may close a loop (the model does not require a radial feeder); opening
 * one may leave buses without supply (the LP is then infeasible and the
 * solve does not converge).  Errors: INVALID_ARG (index, state).          */
int32_t opf_set_line_status(opf_problem* p, int32_t line, int32_t in_service, void* stream, int32_t* n_recomputed);

/* Copy the packed problem to the current CUDA device on `stream`.  With
 * device_arena != NULL the handle carves all its device buffers out of that
 * caller-owned region (>= dims.device_bytes bytes, 256-byte aligned; it must
 * outlive the handle); with NULL it allocates with cudaMallocAsync on
 * `stream` and frees in opf_destroy.  Leaves the state at the initial point
 * of Section V-A.                                                           */
int32_t opf_problem_upload(opf_problem* p, void* device_arena, size_t arena_bytes, void* stream);

/* Run Algorithm 1 on the device until params->criterion holds or
 * params->max_iter iterations have run.  Blocks until the result is known.
 * Returns OPF_OK, OPF_NOT_CONVERGED or an error; *info (may be NULL) gets
 * the residuals of the last check and the objective c^T x in FP64.         */
int32_t opf_admm_solve(opf_problem* p, const opf_params* params, void* stream, opf_info* info);

/* Current iterate in canonical order, copied to caller host buffers (any of
 * them may be NULL): x_global[n_global] (the global vector x), x_local and
 * lam[n_local] (stacked x_s and lambda_s, components in canonical order).
 * Canonical orders: globals = gens (pg, qg per phase), buses (w), loads (pb,
 * qb, pd, qd), in-service lines (p_ij, q_ij, p_ji, q_ji); components =
 * buses, in-service lines, loads, generators; bus locals = w, then for each
 * in-service line touching the bus (line order) the flow leaving the bus
 * (p, q), then its loads' (pb, qb), then its generators' (pg, qg); line
 * locals = p_ij, q_ij, p_ji, q_ji, w_i, w_j; load locals = pb, qb, pd, qd,
 * w; generator locals = pg, qg (each block over the element's phases).    */
int32_t opf_get_state(const opf_problem* p, double* x_global, double* x_local, double* lam,
                      void* stream);

/* Overwrite the local iterate and duals (canonical order, host buffers) for
 * a warm start; the next solve with warm_start = 1 continues from them.    */
int32_t opf_set_state(opf_problem* p, const double* x_local, const double* lam, void* stream);

/* Structure in canonical order (any pointer may be NULL): comp_ptr[S+1]
 * offsets of each component's locals, comp_kind[S] (0 bus, 1 line, 2 load,
 * 3 gen), comp_index[S] (index in the input records), gidx[n_local] (global
 * index of each local copy, i.e. B_s), m_reduced[S] (rows kept by row
 * reduction).                                                               */
int32_t opf_get_structure(const opf_problem* p, int32_t* comp_ptr, int32_t* comp_kind,
                          int32_t* comp_index, int32_t* gidx, int32_t* m_reduced);

/* Unscatter the global vector into per-element arrays (host, caller-owned,
 * 3 doubles per element, NaN for absent phases and out-of-service lines):
 * w[n_bus*3]; pg, qg[n_gen*3]; p_ij, q_ij, p_ji, q_ji[n_line*3];
 * pd, qd, pb, qb[n_load*3].  Any pointer may be NULL.                      */
int32_t opf_get_solution(const opf_problem* p, double* w, double* pg, double* qg,
                         double* p_ij, double* q_ij, double* p_ji, double* q_ji,
                         double* pd, double* qd, double* pb, double* qb, void* stream);

/* Average device duration in microseconds of each kernel of an iteration,
 * as launched inside the solve graph: for each kernel a CUDA graph of
 * `reps` back-to-back launches is timed with CUDA events on `stream`.
 * us[0] = global update, us[1] = local update + dual update (the
 * tile-parallel kernel the graph runs on iterations without residual
 * partials), us[2] = local update with residual partials (the chunk kernel
 * of a check iteration), us[3] = residual finalize.  Uses
 * params->rho and params->precision; the iterate, duals and iteration
 * counter are saved before and restored after (scratch is allocated with
 * cudaMallocAsync on `stream` and freed before returning).                 */
int32_t opf_profile_kernels(opf_problem* p, const opf_params* params, int32_t reps, void* stream, double* us);

/* Per-iteration time of each phase of the shared-memory persistent kernel,
 * in microseconds, measured on the device (globaltimer, thread 0 of each
 * CTA): out[0..3] = mean over CTAs of {global update of the interior halo
 * entries, global update of the boundary entries including the wait for
 * the neighbours' terms and the CTA barrier, local update of the boundary
 * tiles, local update of the interior tiles + CTA barrier + residual
 * check}; out[4..7] = the maximum over CTAs.  Runs `iters` iterations from
 * the initial point (the problem is left at that iterate); needs the
 * shared-memory kernel to fit (else OPF_ERR_INVALID_ARG).                  */
int32_t opf_profile_persistent(opf_problem* p, const opf_params* params, int32_t iters, void* stream, double* out);

/* The same measurement per CTA: per_cta[4*b + k] = microseconds per
 * iteration of phase k (order as above) in chunk b, n_blocks * 4 entries.  */
int32_t opf_profile_persistent_ctas(opf_problem* p, const opf_params* params, int32_t iters, void* stream,
                                    double* per_cta);

/* Layout statistics of each chunk (host data, no device needed), for
 * choosing the chunk count: out[OPF_CHUNK_STATS * b + k] with k =
 * 0 tiles (without padding), 1 interior tiles, 2 operator column groups of
 * four over the chunk's tiles, 3 the largest per-warp sum of (column groups
 * + 2) over the chunk's warps, 4 halo entries, 5 boundary halo entries,
 * 6 copies in the halo lists, 7 copies held by other chunks, 8 neighbour
 * chunks, 9 locals.  The paper has no counterpart.                        */
#define OPF_CHUNK_STATS 10
int32_t opf_chunk_stats(const opf_problem* p, int32_t* out);

/* Engine that OPF_ENGINE_AUTO selects for this problem and precision on the
 * problem's device (OPF_ENGINE_PERSISTENT or OPF_ENGINE_GRAPH).            */
int32_t opf_engine_for(const opf_problem* p, int32_t precision, int32_t* engine);

/* Test and tuning hook (the paper has no counterpart): wait_limit_ns bounds
 * every device-side wait of the persistent engine (default 2e9 ns; a wait
 * that expires makes the solve return OPF_ERR_TIMEOUT with an undefined
 * iterate, and the device stays usable); withhold_block >= 0 makes that CTA
 * never publish its iteration flag, so its neighbours' waits expire (used by
 * the failure-detection test), -1 restores normal operation;
 * persistent_variant selects the persistent kernel: 0 automatic (shared-
 * memory iterate when it fits, else global-memory iterate), 1 global-memory
 * iterate, 2 shared-memory iterate, 3 shared-memory iterate whose boundary
 * terms are polled entry by entry instead of gathered in one pass (same
 * results; OPF_ERR_INVALID_ARG at solve time when 2 or 3 does not fit
 * co-resident).                                                            */
int32_t opf_debug_config(opf_problem* p, int64_t wait_limit_ns, int32_t withhold_block, int32_t persistent_variant);

/* Allocation-free residual norms.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory -- code that
 * runs inside a fixed memory pool that must not grow, plugins that are handed
 * pre-allocated buffers, processes that forbid cudaMalloc after start-up.
 * Inputs are caller-owned device arrays of n_local doubles: v (the global
 * vector gathered per local copy, v_j = x[gidx_j]), x_local and x_local_prev
 * (stacked local copies at this and at the previous iteration), lam (stacked
 * duals).  out is a caller-owned device array of 4 doubles that receives,
 * with 2-norms over all n_local entries,
 *   out[0] = ||v - x_local||,
 *   out[1] = rho * ||x_local - x_local_prev||,
 *   out[2] = eps_rel * max(||v||, ||x_local||),
 *   out[3] = eps_rel * ||lam||.
 * Work is enqueued on `stream`; the call does not synchronize.  No cudaMalloc,
 * cudaFree or allocating routine is called: the per-CTA partial sums live in
 * a fixed 128 KiB array inside the library, which every GPU that loads the
 * library holds until the process exits.  Limit: n_local <= 4,194,304,
 * otherwise OPF_ERR_INVALID_ARG.  The first call in each CUDA context (each
 * device's primary context, or any other context the caller makes current)
 * looks up that array's device address in that context; make it before any
 * stream capture.  All calls share the array: two calls whose work overlaps
 * on the GPU (different streams, or different host threads) race and give
 * wrong results; calls in one stream are ordered and safe.  Each call writes
 * every slot it reads, so no clearing is needed between calls.             */
int32_t opf_residuals_noalloc(const double* v, const double* x_local, const double* x_local_prev,
                              const double* lam, int64_t n_local, double rho, double eps_rel,
                              double* out, void* stream);

/* Host copy of component s's precomputed operator (canonical component
 * order): P[n_s*n_s] row-major = -Abar_s of Eq. (closed_2) (symmetric) and
 * bbar[n_s]; either pointer may be NULL.  *n_s (may be NULL) gets n_s.
 * No device work; valid right after opf_problem_create.                   */
int32_t opf_get_operator(const opf_problem* p, int32_t s, double* P, double* bbar, int32_t* n_s);

/* The precompute of Section IV-B and Eq. (closed_2) applied to caller-given
 * rows: A[m*n] row-major and b[m] (host arrays, read only).  Row reduction
 * keeps a maximal independent subset of the rows (*m_reduced gets its size;
 * may be NULL); P[n*n] row-major receives -Abar_s = I - A^T (A A^T)^{-1} A
 * and bbar[n] receives A^T (A A^T)^{-1} b for the kept rows (either may be
 * NULL).  m = 0 gives P = I, bbar = 0.  Errors: OPF_ERR_INCONSISTENT when a
 * dropped row is not satisfied (the row reduction's 0 = b, b != 0),
 * OPF_ERR_INVALID_ARG for sizes outside [0, 4096] x [1, 4096] or a
 * non-finite entry.  Host only: the same routine opf_problem_create runs on
 * every component of the model.                                            */
int32_t opf_component_operator(const double* A, const double* b, int32_t m, int32_t n, double* P, double* bbar,
                               int32_t* m_reduced);

void opf_destroy(opf_problem* p);

/* ------------------------------------------------------------------ batch
 * Many feeders solved together (the batch dimension of the sweep).  Each
 * instance keeps its own chunks, parameters, iteration counter, residual
 * checks and stopping decision: its iterates do not depend on the other
 * instances in the batch, and are bit-identical to a solve of that problem
 * alone.  params[0].engine picks the engine for the whole batch:
 *   OPF_ENGINE_PERSISTENT  one cooperative launch over every instance's
 *                          chunks; the sum of the chunks must fit
 *                          co-resident (opf_batch_capacity; create the
 *                          problems with opf_problem_create_ex and a chunk
 *                          count sized to the batch), else
 *                          OPF_ERR_INVALID_ARG;
 *   OPF_ENGINE_GRAPH       (HOSTLOOP maps here) a CUDA graph whose while
 *                          node runs one global-update launch and one
 *                          local-update launch per iteration over all
 *                          instances, and the per-instance checks every
 *                          check_every iterations, until every instance has
 *                          stopped; any number of chunks; every entry must
 *                          have the same check_every;
 *   OPF_ENGINE_AUTO        persistent when the chunks fit co-resident,
 *                          except when they fit only with their iterate in
 *                          global memory and the batch's device data is
 *                          larger than the L2 cache (the operators then
 *                          stream from HBM, where the graph engine is
 *                          faster); else graph.
 * All problems must be uploaded on the current device.  The batch borrows
 * the problems (they must outlive it) and owns a small device and
 * pinned-host buffer for the launch descriptors, plus the cached graph.    */
typedef struct opf_batch opf_batch;
int32_t opf_batch_create(opf_problem* const* problems, int32_t n, opf_batch** out);
/* params: n_params == 1 (the same parameters for every instance) or n
 * entries; every entry must have the same precision.  infos: n entries
 * (may be NULL).  Returns OPF_OK when the call ran (per-instance outcomes in
 * infos[i].status) or an error for the whole batch.                       */
int32_t opf_batch_solve(opf_batch* b, const opf_params* params, int32_t n_params, void* stream, opf_info* infos);
void opf_batch_destroy(opf_batch* b);
/* Engine that OPF_ENGINE_AUTO runs for this batch in this precision
 * (OPF_ENGINE_PERSISTENT or OPF_ENGINE_GRAPH), on the batch's device.      */
int32_t opf_batch_engine_for(const opf_batch* b, int32_t precision, int32_t* engine);
/* Chunks (CTAs) that one batch launch can hold co-resident on the current
 * device: the sum of the problems' chunk counts must not exceed it.        */
int32_t opf_batch_capacity(int32_t precision, int32_t* max_chunks);
/* Average device duration in microseconds of each kernel of one iteration
 * of the batched graph engine (the kernels of its while-node body, launched
 * here `reps` times back to back in a plain CUDA graph timed with CUDA
 * events on `stream`): us[0] = global update of every instance, us[1] =
 * local + dual update on the tile-parallel kernel (iterations without
 * residual partials), us[2] = local update with residual partials on the
 * chunk kernel (a check iteration), us[3] = the chunk kernel without
 * partials (for comparison; the body does not run it).  Uses params->rho, params->precision and params->check_every
 * (params[0] for every instance); each instance's iterate, duals, global
 * vector and control block are saved before and restored after (scratch
 * from cudaMallocAsync on `stream`, freed before returning).  The paper has
 * no counterpart: a measurement hook.                                      */
int32_t opf_batch_profile_kernels(opf_batch* b, const opf_params* params, int32_t reps, void* stream, double* us);

/* --------------------------------------------------------------- scenarios
 * Many load scenarios on one feeder topology iterated together (FP32
 * sweeps, FP64 residual sums and objective).  loads holds n_scenarios x
 * n_load records, scenario-major; every scenario's loads must match
 * scenario 0's in bus, phases, connection, alpha and beta (only the draw a,
 * b differs), else OPF_ERR_INVALID_ARG.  Each scenario is Algorithm 1 on
 * its own model: the components that do not depend on the draw share their
 * operator P_s, so their local update (Eq. closed_2) is one small matrix
 * product over all scenarios; load components keep per-scenario bbar_s, and
 * per-scenario P_s where the load is voltage dependent.  Each scenario
 * checks its own residuals and stops at its own check; its iterates are the
 * ones a single-instance FP32 solve of that scenario computes.  Device
 * memory is allocated on the current device at create (cudaMalloc) and
 * freed by destroy.  The paper solves one instance; this is the batch
 * dimension applied to load scenarios.                                     */
typedef struct opf_scenarios opf_scenarios;
int32_t opf_scenarios_create(const opf_bus* buses, int32_t n_bus, const opf_line* lines, int32_t n_line,
                             const opf_gen* gens, int32_t n_gen, const opf_load* loads, int32_t n_load,
                             int32_t n_scenarios, opf_scenarios** out);
/* params: precision must be OPF_FP32, adaptive_rho 0 and check_every in
 * [1, 4096] (the solve graph holds that many iterations of kernel nodes);
 * warm_start continues every scenario from its current state.  infos: n_scenarios entries (may
 * be NULL); status per scenario as for opf_admm_solve.                     */
int32_t opf_scenarios_solve(opf_scenarios* sc, const opf_params* params, void* stream, opf_info* infos);
/* State of one scenario in the canonical orders (host, caller-owned; any
 * pointer may be NULL): x[n_global], xl[n_local], lam[n_local].            */
int32_t opf_scenarios_get_state(const opf_scenarios* sc, int32_t scenario, double* x, double* xl, double* lam,
                                void* stream);
int32_t opf_scenarios_dims(const opf_scenarios* sc, int32_t* n_global, int32_t* n_local, int64_t* device_bytes);
/* Average device time in microseconds of each kernel of one iteration, each
 * launched `reps` times back to back outside the solve graph: us[0] global
 * update, us[1] local update of components with at most 8 locals, us[2] of
 * the larger ones, us[3] both local updates on a check iteration, us[4] the
 * per-scenario check.  Uses params->rho; leaves the scenarios at a cold
 * start.                                                                   */
int32_t opf_scenarios_profile(opf_scenarios* sc, const opf_params* params, int32_t reps, void* stream, double* us);
/* Arithmetic of the local update of Eq. (closed_2) for the components with
 * at most 8 locals whose operator P_s is shared by every scenario (buses,
 * lines, generators, constant-power loads): for 64 scenarios at a time it
 * is the small matrix product X_s = P_s U_s + bbar_s.
 *   OPF_SC_XUPDATE_CUDA_CORES (default): packed FP32 fmas, the operation
 *     order of the single-instance engines, so each scenario's iterates are
 *     bit-identical to solving it alone in FP32;
 *   OPF_SC_XUPDATE_TENSOR: tensor cores (mma.sync m16n8k8, TF32 inputs,
 *     FP32 accumulation) with each operand split into two TF32 parts and
 *     three products (hi*hi + hi*lo + lo*hi), about FP32 accuracy but not
 *     the same bits; used on the iterations between residual checks (a
 *     check iteration and the per-scenario operators of voltage-dependent
 *     loads keep the CUDA-core path).
 * Takes effect at the next opf_scenarios_solve.  INVALID_ARG otherwise.   */
enum { OPF_SC_XUPDATE_CUDA_CORES = 0, OPF_SC_XUPDATE_TENSOR = 1 };
int32_t opf_scenarios_set_xupdate(opf_scenarios* sc, int32_t kind);
void opf_scenarios_destroy(opf_scenarios* sc);

/* ----------------------------------------------------------------- serving
 * Continuous batching: requests (feeders) are submitted at any time; each
 * opf_server_step collects the round in flight, retires finished instances,
 * admits queued requests in arrival order while a slot, the device memory
 * budget and the co-resident chunk capacity allow (finished instances stay
 * resident for warm starts and are evicted least recently used first), and
 * launches the next round asynchronously: round_iters iterations of one
 * batch launch over every active instance.  Host-side model building and
 * precompute (in submit) and uploads (in step, on a side stream) overlap the
 * round running on the device.  A request with warm_from = id of a finished
 * resident request starts from that feeder's iterate for every local copy
 * whose component and global variable are unchanged (a topology switch);
 * when the budget cannot hold both and nothing else is active or
 * evictable, the source is evicted and the request starts cold.
 * Rounds are whole multiples of params.check_every and all engines compute
 * bit-identical iterates, so a request's result does not depend on the mix.
 * Not thread-safe across steps; submit may be called between steps.        */
typedef struct opf_server opf_server;

typedef struct opf_server_config {
    int64_t device_budget_bytes;  /* resident instance arenas stay below this   */
    int32_t max_active;           /* instances iterated per round                */
    int32_t round_iters;          /* iterations per round, multiple of check_every */
    int32_t max_chunks;           /* CTAs per round (0: the device's batch capacity,
                                     opf_batch_capacity)                         */
    int32_t iters_per_bus;        /* iteration budget per bus of a request: its
                                     budget is max(params.max_iter, iters_per_bus
                                     x n_bus); 0 = params.max_iter for all       */
    int32_t _reserved[2];
    opf_params params;            /* solve parameters of every request; max_iter
                                     is each request's iteration budget (see
                                     iters_per_bus)                              */
} opf_server_config;

typedef struct opf_server_stats {
    int64_t submitted, admitted, completed, converged, warm_started, evicted, rounds, iterations;
    int64_t resident_bytes;
    int32_t active, pending;
} opf_server_stats;

void opf_server_config_default(opf_server_config* c);  /* FP32, rho 10, ABS 1e-4, 8 GiB */
int32_t opf_server_create(const opf_server_config* cfg, opf_server** out);
/* chunks <= 0: one chunk per 50 buses (1..64).  *id receives the request id. */
int32_t opf_server_submit(opf_server* s, const opf_bus* buses, int32_t n_bus, const opf_line* lines, int32_t n_line,
                          const opf_gen* gens, int32_t n_gen, const opf_load* loads, int32_t n_load,
                          int32_t chunks, int64_t warm_from, int64_t* id);
int32_t opf_server_step(opf_server* s, void* stream, int32_t* n_active, int32_t* n_pending);
/* Finished requests since the last poll: ids[k], infos[k] (infos[k].seconds =
 * latency from submit to the end of the round that finished it).          */
int32_t opf_server_poll(opf_server* s, int64_t* ids, opf_info* infos, int32_t cap, int32_t* n);
/* The resident problem of a finished request (borrowed; valid until it is
 * evicted or the server is destroyed): use opf_get_solution / opf_get_state. */
int32_t opf_server_problem(opf_server* s, int64_t id, opf_problem** p);
int32_t opf_server_get_stats(opf_server* s, opf_server_stats* stats);
void opf_server_destroy(opf_server* s);

#ifdef __cplusplus
}
#endif
#endif /* OPF_ADMM_H */
