/*
 * hfav.h -- C ABI of the GB300-native HFAV library (libhfav.so).
 *
 * HFAV (Sewall & Pennycook, "High-Performance Code Generation through Fusion
 * and Vectorization", arXiv 1710.08774) takes axioms (terminal inputs), goals
 * (terminal outputs) and production rules (kernels with the relative stencil
 * offsets they read, Sec. 1.1 and the YAML listing of Sec. 4), infers the
 * dataflow DAG (Sec. 3.2), fuses the iteration nests (Sec. 3.3, Listings
 * "fuse_inest_dag" / "fuse_inest"), splits at reduction-to-broadcast dataflow
 * (Sec. 3.4 "Splits"), sizes every variable by the Minkowski sum of its
 * offsets and contracts intermediates into rolling buffers (Sec. 3.5), and
 * emits fused loop nests.  This library does the analysis on the host and
 * runs the fused pipelines as hand-written sm_103a kernels that keep the
 * rolling buffers in registers or shared memory.
 *
 * Conventions for every entry point:
 *   - Return value: HFAV_OK (0) on success, a negative HFAV_E* code on error,
 *     a positive HFAV_WARN_* code when the run completed with a warning.
 *     On any non-zero return hfav_last_error() holds a one-line message
 *     (thread-local, valid until the next call on the same thread).
 *   - Device pointers are plain CUDA device addresses (e.g. a torch tensor's
 *     data_ptr()); the caller owns them and keeps them alive until the work
 *     queued on the given stream has finished.  Host pointers are read during
 *     the call only.
 *   - Streams are cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  All device work is asynchronous on that stream unless stated.
 *   - Arrays are row-major with axis 0 (i) contiguous: element (i, j, k) of a
 *     grid sits at ptr[(k + h) * pitch[2] + (j + h) * pitch[1] + (i + h)],
 *     h = the grid's halo; pitches are in elements.
 */
#ifndef HFAV_H
#define HFAV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif
#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define HFAV_OK 0
#define HFAV_WARN_NEWTON 1       /* some Riemann Newton loops hit the 10-iteration cap */
#define HFAV_EINVAL -1           /* bad argument (null pointer, bad size, bad op id ...) */
#define HFAV_ECYCLE -2           /* the rule DAG has a cycle (Sec. 3.2 requires a DAG) */
#define HFAV_EPRODUCER -3        /* a field has two producers (Sec. 2: one producer per output) */
#define HFAV_EMISSING -4         /* a rule input is neither an axiom nor produced by a rule */
#define HFAV_EHALO -5            /* grid halo / pitch smaller than the inferred footprint */
#define HFAV_EALIGN -6           /* pointer or pitch not 16-byte aligned */
#define HFAV_ENOMEM -7           /* device or host allocation failed */
#define HFAV_ECUDA -8            /* a CUDA runtime call failed */
#define HFAV_ETIMEOUT -9         /* a bounded device wait gave up */
#define HFAV_ENONPHYSICAL -10    /* negative density or pressure produced (CFL too large) */
#define HFAV_EUNSUPPORTED -11    /* valid DAG but no kernel for this op / schedule */

/* ---- element types --------------------------------------------------- */
typedef enum {
    HFAV_F64 = 0,   /* every value and every operation in FP64 */
    HFAV_F32 = 1    /* fields and bulk arithmetic in FP32; the Riemann Newton
                       iteration for p* and the CFL reduction in FP64 */
} hfav_dtype;

/* ---- boundary handling (the make_boundary kernel of Hydro2D, Sec. 5.4) - */
typedef enum {
    HFAV_BC_PERIODIC = 0,    /* halo cells are never read; indices wrap onto the interior */
    HFAV_BC_HALO_GIVEN = 1   /* the caller fills the axioms' halo; it is read as given */
} hfav_bc;

/* ---- builtin rule catalogue ----------------------------------------- */
/* Every op's inputs are listed in the order given here.  "Directional" ops
 * act along rule.axis; their offsets in hfav_ref must be along that axis. */
typedef enum {
    /* out = sum_k params[k] * in[k]                    (any refs, n_params == n_in) */
    HFAV_OP_STENCIL_LINEAR = 1,
    /* out = sqrt(sum_d (in[2d] - in[2d+1])^2) / 2      (n_in even, params none)     */
    HFAV_OP_GRADMAG_HALF = 2,
    /* out = in / (1 + in)                              (1 ref)                       */
    HFAV_OP_SQUASH = 3,
    /* generic pointwise ops used by planner-only examples (not run on the GPU)       */
    HFAV_OP_GENERIC = 4,
    /* COSMO horizontal diffusion (Sec. 5.3 names its kernels flux_x / flux_y and
     * ustage; the first, ulapstage, is a STENCIL_LINEAR 5-point star):
     * LIMFLUX, directional along rule.axis, in: u(0) u(+1) lap(0) lap(+1)
     *   f = lap(+1) - lap(0); out = 0 where f (u(+1) - u(0)) > 0, else f
     *   (the flux of the face +1/2, stored at index 0)
     * DIFFUSE, in: u flx(-1,0) flx(0) fly(0,-1) fly(0), params[0] = c
     *   out = u - c ((flx(0) - flx(-1)) + (fly(0) - fly(-1)))                          */
    HFAV_OP_LIMFLUX = 5,
    HFAV_OP_DIFFUSE = 6,
    /* A user rule body (the paper's rules name arbitrary kernels, Sec. 1.1 and
     * the rule listing of Sec. 4): rule.expr is a C expression giving the one
     * output from in0 .. in{n_in-1} (the inputs at their offsets) and
     * p0 .. p{n_params-1} (the parameters), evaluated in the plan's precision
     * (type T: double for HFAV_F64, float for HFAV_F32) with the CUDA math
     * functions (sqrt, fabs, fmin, fmax, exp, ...) and the ?: operator.  The
     * plan generates, compiles (NVRTC, at the first run on a device) and
     * caches the kernels.  Rejected at plan creation (HFAV_EINVAL): characters
     * outside [A-Za-z0-9_ .+-*<>/%()!=&|?:,^~], a single '&', comments, names
     * in<k> / p<k> beyond the rule's inputs / parameters, and any other name
     * but T, double, float, int and the math functions sqrt rsqrt cbrt exp
     * exp2 expm1 log log2 log10 log1p pow sin cos tan asin acos atan atan2
     * sinh cosh tanh asinh acosh atanh fabs fmin fmax fma floor ceil trunc
     * round rint copysign fmod hypot erf erfc tgamma lgamma fdim -- so a body
     * reads nothing but its inputs.  An expression that does not compile fails
     * the run with HFAV_EINVAL and the compiler log in hfav_last_error(). */
    HFAV_OP_EXPR = 7,
    /* Hydro2D kernels (Sec. 5.4), directional, ideal gas, params[0] = gamma:
     * CONSTOPRIM in: U0 U1 U2 U3 (rho, rho u, rho v, E) -> rho un ut e
     * EOS        in: rho e                              -> p c
     * SLOPE      in: q(-1) q(0) q(+1) for rho un ut p   -> drho dun dut dp
     * TRACE      in: rho un ut p c drho dun dut dp dt   -> qm[4] qp[4]
     * QLEFTRIGHT in: qp[4](0) qm[4](+1)                 -> qL[4] qR[4]
     * RIEMANN    in: qL[4] qR[4]                        -> g[4]
     *            (params[1], optional: cap on the Newton iterations, 1..10,
     *            default 10; faces that reach it are counted and reported
     *            as HFAV_WARN_NEWTON)
     * CMPFLX     in: g[4]                               -> F[4]
     * UPDATE     in: U0..U3 F[4](0) F[4](-1) dt         -> U'0..U'3
     * The face a+1/2 is stored at index a. */
    HFAV_OP_CONSTOPRIM = 10,
    HFAV_OP_EOS = 11,
    HFAV_OP_SLOPE = 12,
    HFAV_OP_TRACE = 13,
    HFAV_OP_QLEFTRIGHT = 14,
    HFAV_OP_RIEMANN = 15,
    HFAV_OP_CMPFLX = 16,
    HFAV_OP_UPDATE = 17,
    /* reduction: dt = params[0] * dx / max over interior cells of max(|u|+c, |v|+c)
     * in: U0 U1 U2 U3; out: one rank-0 field; params: cfl, gamma */
    HFAV_OP_CFL_DT = 20,
    /* reductions (Sec. 3.4), in: one grid field (any offset); out: one rank-0
     * field = the sum / the maximum of the input over the interior cells,
     * accumulated in FP64.  Rule bodies (HFAV_OP_EXPR) over rank-0 inputs
     * finalize such results (e.g. a root); a rule body over the grid reads a
     * rank-0 field at offset 0 as one value (a broadcast), next to at least one
     * grid field.  A rank-0 field is neither an axiom nor a goal.  Such DAGs run on generated kernels, 2D
     * only: the fused form is one kernel per fusion group (the reduction
     * splits the DAG), the unfused form one kernel per rule; the partials of
     * each reduction are combined in a fixed order (bitwise repeatable). */
    HFAV_OP_REDUCE_SUM = 21,
    /* planner-only broadcast op of the analysis examples */
    HFAV_OP_BROADCAST = 22,
    HFAV_OP_REDUCE_MAX = 23
} hfav_op;

/* A reference to a field at a relative offset (i, j, k): the paper's
 * translation-free description of a kernel argument (Sec. 3.1), e.g. q?[j?-1][i?]. */
typedef struct {
    int field;
    int off[3];
} hfav_ref;

/* A production rule: one kernel callsite group (Sec. 3.2.2 "Grouping"). */
typedef struct {
    int op;                  /* hfav_op */
    int axis;                /* sweep axis of directional ops, else 0 */
    int n_in;
    const hfav_ref* in;
    int n_out;
    const int* out;          /* field ids written at offset 0 */
    int n_params;
    const double* params;
    const char* expr;        /* HFAV_OP_EXPR: the rule body (NUL-terminated, at
                                most 4096 characters, read during plan creation);
                                NULL for the other ops */
} hfav_rule;

/* The rule DAG.  Field ranks: ndim for grid fields, 0 for scalars (the result
 * of a reduction, e.g. the CFL time step). */
typedef struct {
    int n_fields;
    const int* field_rank;
    int n_rules;
    const hfav_rule* rules;
    int n_axioms;
    const int* axioms;       /* terminal inputs, caller-owned arrays */
    int n_goals;
    const int* goals;        /* terminal outputs, caller-owned arrays */
    int ndim;                /* 1, 2 or 3 */
    int stream_axis;         /* outermost loop axis of the fused nest (global loop order) */
    int feedback;            /* 1: goal g is the next time level of axiom g (time stepping) */
    /* Declared in/out aliasing (Sec. 3.5 "In/out chaining"): NULL, or n_goals
     * entries, inout[g] = the index in `axioms` of the axiom whose array goal g
     * may share (an in-place update), -1 for none.  The result is the one the
     * non-aliased run gives.  Not with feedback; each axiom at most once. */
    const int* inout;
} hfav_dag;

/* One grid: interior extents, allocation pitches and halo width of every
 * axiom / goal array of that grid.  Unused axes have extent 1. */
typedef struct {
    int64_t extent[3];
    int64_t pitch[3];        /* pitch[0] must be 1 */
    int halo;
} hfav_grid;

/* Storage class the planner assigns to a field (Sec. 3.5). */
typedef enum {
    HFAV_STORE_AXIOM = 0,    /* caller array in HBM */
    HFAV_STORE_GOAL = 1,     /* caller array in HBM */
    HFAV_STORE_HBM = 2,      /* full plan-owned array: its enclosing region spans nests */
    HFAV_STORE_ROLLING = 3,  /* contracted rolling buffer inside one fused nest */
    HFAV_STORE_SCALAR = 4    /* rank-0 value (reduction result) */
} hfav_storage;

/* Per-field result of the analysis. */
typedef struct {
    int producer;            /* rule id, -1 for axioms */
    int group;               /* fusion group of the producer, -1 for axioms */
    int storage;             /* hfav_storage */
    int halo_lo[3];          /* cells needed below the goal region, per axis */
    int halo_hi[3];          /* cells needed above the goal region, per axis */
    int window[3];           /* span of the field's composed offsets per axis (Sec. 3.5 "Contraction") */
    int stage_window[3];     /* span of the direct consumers' offsets per axis */
    int64_t storage_elems;   /* rolling-buffer elements: window along the outermost
                                axis with span > 1 times the inner interior extents */
    int n_reuse;             /* number of distinct offsets in the reuse order */
    int reuse[27][3];        /* offsets in order of first to last use (Sec. 3.5 "Grouping") */
} hfav_field_info;

/* Statistics of the last hfav_run (hfav_status synchronises the plan's stream). */
typedef struct {
    int64_t newton_nonconverged;   /* faces whose Newton loop hit the cap */
    int64_t nonphysical;           /* cells with rho <= 0 or p <= 0 after an update */
    int n_dt;                      /* entries written to dt[] (steps of grid 0) */
    double dt[64];                 /* time steps of grid 0, first 64 steps */
    double last_ms;                /* device time of the last run (CUDA events) */
    int last_launches;             /* kernels launched by the last run */
} hfav_run_stats;

typedef struct hfav_plan_s hfav_plan_t;

/* ---- planning -------------------------------------------------------- */

/*
 * hfav_plan: validate the DAG, order it topologically (Sec. 3.2), infer every
 * field's footprint and halo (Sec. 3.5, Minkowski sum of offsets), fuse the
 * iteration nests and find splits (Sec. 3.3, 3.4), contract intermediates
 * (Sec. 3.5), map each fusion group onto a kernel pipeline and pick a schedule.
 *   dag       : the rule DAG (copied; may be freed after the call).
 *   grids     : n_grids grid descriptions (copied).  Every axiom/goal array of
 *               grid g uses grids[g]'s extents, pitches and halo.
 *   dtype     : hfav_dtype.  bc: hfav_bc.
 *   schedule  : NULL or "auto" (default schedule), "tuned" (hfav_autotune on
 *               the arrays of the first hfav_run / hfav_run_graph, which then
 *               runs the fastest variant), or an explicit variant
 *               "<fusion>[:<placement>][:<TX>x<TY>]" with fusion in
 *               {full, sweep, unfused}, placement in {reg, smem, hbm}.
 *               Generated kernels (DAGs with rule bodies or reductions) in
 *               2D take full:smem (rows in shared-memory rings), full:reg
 *               (warp strips, rows in registers: one fused part without
 *               reductions, reads within 4 cells (FP32) / 2 (FP64) in x;
 *               otherwise EUNSUPPORTED with the reason) or unfused.
 *               When schedule is NULL or "auto" and the environment variable
 *               HFAV_SCHEDULE is set, its value ("auto", "tuned" or a variant)
 *               is used instead.
 *   out       : receives the plan; release with hfav_free.
 * Host only: no device memory is touched until the first hfav_run.
 * Errors: EINVAL, ECYCLE, EPRODUCER, EMISSING, EHALO, EUNSUPPORTED, ENOMEM.
 */
int hfav_plan(const hfav_dag* dag, const hfav_grid* grids, int n_grids, int dtype, int bc,
              const char* schedule, hfav_plan_t** out);

/* Analysis only (no grids, no schedule): the same validation, footprint,
 * fusion and contraction as hfav_plan.  extent gives the interior extents
 * used for storage sizes (may be NULL: extents of 1). */
int hfav_analyze(const hfav_dag* dag, const int64_t* extent, hfav_plan_t** out);

/* Number of fusion groups and the group of each rule (array of n_rules). */
int hfav_plan_groups(const hfav_plan_t* plan, int* n_groups, int* rule_group, int n_rules);

/* Analysis result for one field. */
int hfav_plan_field(const hfav_plan_t* plan, int field, hfav_field_info* info);

/* Topological rule order (array of n_rules). */
int hfav_plan_order(const hfav_plan_t* plan, int* order, int n_rules);

/* Replace the schedule (same grammar as hfav_plan).  Drops any captured graph. */
int hfav_plan_set_schedule(hfav_plan_t* plan, const char* schedule);

/* Current schedule as a string "<fusion>:<placement>:<TX>x<TY>". */
int hfav_plan_schedule(const hfav_plan_t* plan, char* buf, size_t n);

/* JSON dump of the analysis: groups, order, per-field footprint, windows, storage. */
int hfav_plan_dump(const hfav_plan_t* plan, char* buf, size_t n);

/* The CUDA C++ source of the kernels a plan of generated kernels (a DAG
 * with HFAV_OP_EXPR rules or reductions) compiles under its current
 * schedule -- the emitted code of the method (Sec. 3.6): one streaming or
 * pointwise kernel per fusion group (fused) or per rule (unfused), and a
 * finalization kernel after each part with reductions.  Each separately
 * compiled unit follows a line starting with "// ---- kernel".  Copies up to
 * n - 1 characters and a NUL into buf; HFAV_EINVAL (message: the size
 * needed) when buf is too small, HFAV_EUNSUPPORTED for plans of the builtin
 * kernels.  Needs no device. */
int hfav_plan_source(const hfav_plan_t* plan, char* buf, size_t n);

/* Features of the plan under a schedule for the learned cost model: writes
 * HFAV_N_FEATURES floats (DAG depth, stencil radius, field count, log cells,
 * dtype, fusion, placement, tile, compulsory bytes, recompute ratio ...). */
#define HFAV_N_FEATURES 16
/* feature HFAV_FEATURE_BASE holds log2(analytic time estimate in us) / 16;
 * the learned model predicts ln(time) minus ln of that estimate */
#define HFAV_FEATURE_BASE 12
int hfav_plan_features(const hfav_plan_t* plan, const char* schedule, float* feat);

/* ---- execution ------------------------------------------------------- */

/*
 * hfav_run: run the plan n_steps times on `stream`.
 *   axiom_ptrs: n_grids * n_axioms device pointers, grid-major, in dag.axioms order.
 *   goal_ptrs : n_grids * n_goals device pointers, grid-major, in dag.goals order.
 *   n_steps   : >= 1; with dag.feedback the goals of step s are the axioms of
 *               step s+1 (the plan ping-pongs through its own scratch so the
 *               axiom arrays are never written and the last step lands in
 *               the goal arrays); without feedback n_steps must be 1.
 * A goal pointer may equal an axiom pointer only where dag.inout declares
 * it; any other overlap of goals and axioms is refused (HFAV_EINVAL).  For a
 * declared in-place run the plan copies the axiom values the update still
 * needs to temporaries first (Sec. 3.5 "In/out chaining"): the generated
 * fused 2D kernels save only the halo bands at their CTA boundaries (a few
 * rows and columns per CTA), every other pipeline the whole axiom array
 * (plan-owned).  The halo cells of goal arrays are left unspecified.
 * Plan-owned scratch (ping-pong state, HBM intermediates of split or unfused
 * schedules, per-grid time-step slots, counters) is allocated on first use and
 * kept until hfav_free.  Asynchrony: a run that allocates (the plan's first
 * run, or one that needs a larger scratch buffer) synchronises the device
 * through cudaMalloc; otherwise the call queues its table uploads (ordered
 * copies from host memory that may be reused once the call returns) and its
 * kernels on `stream` and returns without waiting for the GPU, so runs queued
 * back to back on one stream, each reading the previous one's goals, are
 * ordered correctly.  The runs of one plan share its scratch: queue them on
 * one stream, or order the streams yourself.
 * Errors: EINVAL, EALIGN, ENOMEM, ECUDA.  Newton / non-physical results are
 * reported by hfav_status, which synchronises.
 */
int hfav_run(hfav_plan_t* plan, void* const* axiom_ptrs, void* const* goal_ptrs, int n_steps,
             void* stream);

/* Same as hfav_run, but the whole n_steps sequence is captured once into a
 * CUDA graph (per plan, keyed on the pointers, n_steps, schedule and stream)
 * and replayed.  The uncaptured preparation run before a capture works on
 * plan-owned copies of in-place (dag.inout) arrays, so each call updates them
 * exactly once.  The graph uploads its own pointer tables from pinned host
 * memory that nothing else writes, so plain hfav_run calls between replays
 * (on other arrays) leave it intact; a plain run that has to grow a scratch
 * buffer drops the graph (after its last replay finishes) and the next
 * hfav_run_graph captures a new one.  Building a graph synchronises `stream`. */
int hfav_run_graph(hfav_plan_t* plan, void* const* axiom_ptrs, void* const* goal_ptrs, int n_steps,
                   void* stream);

/* Synchronise the plan's last stream and read its counters and dt history.
 * Returns HFAV_OK, HFAV_WARN_NEWTON, or HFAV_ENONPHYSICAL. */
int hfav_status(hfav_plan_t* plan, hfav_run_stats* stats);

/*
 * hfav_autotune: time every valid schedule of the plan (fusion x placement x
 * tile) on the given arrays with CUDA events (median of `reps` after one warm
 * run), keep the fastest as the plan's schedule.  times_ms receives one time
 * per variant in the order of hfav_plan_variants (may be NULL).  In-place
 * (dag.inout) arrays are timed on plan-owned copies and left unchanged.
 */
int hfav_autotune(hfav_plan_t* plan, void* const* axiom_ptrs, void* const* goal_ptrs, int n_steps,
                  int reps, void* stream, float* times_ms, int n_times);

/* Valid schedule strings of the plan, '\n'-separated; returns the count. */
int hfav_plan_variants(const hfav_plan_t* plan, char* buf, size_t n);

/* Per-kernel timing: when enabled, every later hfav_run records a CUDA event
 * after each kernel launch (not inside a captured graph).  hfav_kernel_times
 * synchronises on the last event and writes, per distinct kernel of the last
 * run, its name ('\n'-separated into names), total device time (ms, the time
 * between the events that bracket each launch on the stream) and launch
 * count.  Returns the number of kernels. */
int hfav_plan_timing(hfav_plan_t* plan, int enable);
int hfav_kernel_times(hfav_plan_t* plan, char* names, size_t n_names, double* ms, int* counts, int max_kernels);

/*
 * hfav_chain2d_static: the 2D three-stage chain (L = weighted 5-point star of u,
 * G = |central gradient of L| / 2, out = G / (1 + G)) computed without any
 * device allocation, for callers that cannot allocate device memory once they
 * are running (a host application whose pool owns the device's memory, a
 * latency-critical loop that must avoid cudaMalloc's implicit synchronisation,
 * a caller without a plan).  The paper has no counterpart: it is a deployment
 * variant of the chain's "sweep" schedule, whose materialised L lives here in a
 * file-scope device array of HFAV_STATIC_SCRATCH_BYTES = 16 MiB instead of a
 * plan-owned buffer.
 *   u, out   : device arrays of the same layout: (ny + 2 halo) rows of pitch
 *              elements, interior at (halo, halo); out's halo is not written.
 *   bc       : HFAV_BC_PERIODIC (halo never read) or HFAV_BC_HALO_GIVEN
 *              (halo >= 2, read as given).
 *   weights  : host array of 5 weights of u(i+1), u(i-1), u(j+1), u(j-1),
 *              u(i, j), or NULL for (1, 1, 1, 1, -4).
 *   stream   : cudaStream_t (NULL = legacy stream); asynchronous.
 * Limits and behaviour: (nx + 2) * (ny + 2) * 8 bytes must fit the 16 MiB
 * array, else HFAV_EINVAL and no device work; u and out must not overlap
 * (HFAV_EINVAL).  With CUDA's default lazy module loading the array is
 * reserved on a device by the first call made there, which also looks up its
 * address on that device: make that first call at start-up, before any stream
 * capture and before a memory pool takes the device's remaining memory (if
 * 16 MiB are no longer free it fails with HFAV_ENOMEM).  From then on the
 * device holds the array until the process exits.  The address is cached per
 * device for the life of the process, so the call must not be used across a
 * cudaDeviceReset.  All calls share the array and each overwrites all of L it
 * reads; calls whose device work overlaps race.  Allocates nothing (no
 * cudaMalloc, cudaFree or allocating library call).
 */
int hfav_chain2d_static(const double* u, int64_t nx, int64_t ny, int64_t pitch, int halo, int bc,
                        const double* weights, double* out, void* stream);

/* Diagnostic: the FP64 reciprocal and quotient the Godunov kernels use in
 * place of IEEE division (hardware estimate refined by two Newton-Raphson
 * steps; quotient with one residual correction).  For n doubles x (device):
 * rcp_out[k] = 1/x[k], quot_out[k] = 1.5/x[k] (device arrays).  Tests hold
 * them to within 2 ulp of IEEE division. */
int hfav_selftest_arith(const double* x, int64_t n, double* rcp_out, double* quot_out, void* stream);

/* Diagnostic: the FP64 reciprocal square root of the Riemann solver's Newton
 * iteration in the FP32-bulk form (hardware estimate refined by one
 * Newton-Raphson step).  For n positive doubles x (device): out[k] ~
 * 1/sqrt(x[k]) (device array).  Tests hold it to within 2^-38 relative of
 * CUDA's rsqrt. */
int hfav_selftest_rsqrt(const double* x, int64_t n, double* out, void* stream);

/* Diagnostic: the halving of the Godunov kernels' FP64 arithmetic, done on the
 * integer pipe (exponent field lowered by one; zeros unchanged; results that
 * would be subnormal, infinities and NaNs through the FP64 multiply).  For n
 * doubles x (device): out[k] = x[k] / 2 (device array).  Tests hold it bit for
 * bit to the IEEE product x * 0.5 (NaNs: NaN). */
int hfav_selftest_half(const double* x, int64_t n, double* out, void* stream);

/* Diagnostic: the FP64 <-> FP32 conversions of the FP32-bulk Riemann solver,
 * done on the integer pipe (exponent rebiased, significand shifted; the
 * narrowing rounds to nearest even; zeros, subnormals, infinities and NaNs
 * through the conversion instructions).  For n doubles x and n floats f
 * (device): narrow_out[k] = (float)x[k], widen_out[k] = (double)f[k] (device
 * arrays).  Tests hold both bit for bit to the IEEE conversions. */
int hfav_selftest_convert(const double* x, const float* f, int64_t n, float* narrow_out, double* widen_out,
                          void* stream);

/* Diagnostic: measured arithmetic peaks of the current device, the
 * denominators of the ALU rooflines.  Writes rates[0] = FP64 fused
 * multiply-adds per second (one per thread per instruction, the FP64 pipe's
 * issue rate), rates[1..3] = FP64 IEEE divides, square roots and CUDA
 * reciprocal square roots per second, rates[4] = FP32 fused multiply-adds per
 * second, each from eight independent dependency chains per thread on 8 CTAs
 * of 256 threads per SM, timed with CUDA events on `stream` after a warm-up
 * launch (about 0.1 s of device time; synchronises).  The ratio
 * rates[0] / rates[k] is the cost of operation k in FP64 pipe slots.  n must
 * be >= 5.  The paper has no counterpart. */
int hfav_probe_peaks(double* rates, int n, void* stream);

/* Fault injection for tests of the failure paths: after `after` more device
 * allocations by the library (plan scratch, counters, model buffers), the
 * next one fails once as if the device were out of memory, and the call that
 * made it returns HFAV_ENOMEM with the plan left usable; after < 0 turns the
 * injection off.  Process-wide, host only; returns HFAV_OK.  The paper has no
 * counterpart. */
int hfav_inject_alloc_failure(int after);

void hfav_free(hfav_plan_t* plan);

const char* hfav_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int hfav_version(void);

/* ---- learned schedule model (small MLP, FP32, own CUDA kernels) ---------
 * Network: n_in -> H -> H -> 1 with ReLU, H = hidden.  Parameters live in one
 * device array laid out [W1 (H x n_in), b1 (H), W2 (H x H), b2 (H), w3 (H), b3 (1)],
 * row-major, size hfav_mlp_n_params(n_in, hidden). */
int64_t hfav_mlp_n_params(int n_in, int hidden);

/* y[n] = f(X[n x n_in]) for device arrays.  hidden <= 128. */
int hfav_mlp_forward(const float* params, int n_in, int hidden, const float* X, int n, float* y,
                     void* stream);

/* Mean squared error over n rows and its gradient w.r.t. params (device
 * arrays; grad has n_params floats, loss one float).  work must hold
 * hfav_mlp_work_floats(n, hidden) floats of caller-owned device scratch. */
int64_t hfav_mlp_work_floats(int n, int hidden);
int hfav_mlp_loss_grad(const float* params, int n_in, int hidden, const float* X, const float* t,
                       int n, float* grad, float* loss, float* work, void* stream);

/* One Adam step (Kingma & Ba 2015) on device arrays; step is 1-based. */
int hfav_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t n_params,
                  float lr, float beta1, float beta2, float eps, int step, void* stream);

/* Full-batch training: `epochs` steps of (loss_grad, adam) with lr and Adam's
 * default betas (0.9, 0.999) and eps 1e-8.  params, m, v: device arrays of
 * n_params floats (m, v zeroed by the caller before the first call); work and
 * grad as for hfav_mlp_loss_grad; loss_hist: device array of `epochs` floats
 * receiving the loss before each step. */
int hfav_mlp_train(float* params, float* m, float* v, int n_in, int hidden, const float* X, const float* t, int n,
                   int epochs, float lr, float* work, float* grad, float* loss_hist, void* stream);

/* Learned schedule choice: features of every valid schedule of the plan
 * (hfav_plan_features, then (f - shift) * scale per feature when the host
 * arrays are given), the predicted ln(time) of each -- the mean output of the
 * n_models networks whose parameter vectors lie back to back in `params`
 * (device), plus ln of the analytic estimate in feature HFAV_FEATURE_BASE --
 * (pred, host, n_pred entries in hfav_plan_variants order), and the argmin
 * installed as the plan's schedule and copied to `best`.  Synchronises the
 * default stream. */
int hfav_model_choose(hfav_plan_t* plan, const float* params, int n_models, int hidden, const float* feat_shift,
                      const float* feat_scale, float* pred, int n_pred, char* best, size_t n_best);

#ifdef __cplusplus
}
#endif
#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#endif /* HFAV_H */
