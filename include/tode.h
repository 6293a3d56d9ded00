/*
 * tode.h -- C ABI of the B300 batched adaptive Dormand-Prince 5(4) solver.
 *
 * The library solves B independent initial value problems y' = f(t, y),
 * each with its own initial state, integration range, step size, error
 * estimate, accept/reject decisions and evaluation times (torchode, Sec. 3:
 * the solver keeps a separate state per instance; Sec. 4.1 shows why
 * instances must not share a step size).  The method is dopri5 (App. A) with
 * FSAL/SSAL and Horner dense output (Sec. 3, "What makes torchode fast?"),
 * a PI step-size controller of Soderlind's family (Sec. 3, App. C) and per-
 * instance statistics and status (Sec. 3; App. B).
 *
 * Conventions for every entry point:
 *  - Pointers are DEVICE pointers unless marked "host".  The caller owns and
 *    allocates every buffer (inputs, outputs, workspace, tape, scratch); the
 *    library never allocates or frees device memory and calls no library
 *    that does.
 *  - Calls enqueue work on `stream` (a cudaStream_t, NULL = legacy default)
 *    and return.  Outputs are valid once the stream has synchronised.  The
 *    plain form (TODE_PLAIN) additionally synchronises `stream` every
 *    `poll_every` steps to read its "any instance still running" flag.
 *  - Argument and launch errors are returned as tode_err before or at launch
 *    and leave outputs unspecified.  Numerical failures never abort the
 *    batch: they are reported per instance in status[].
 *  - Times (t0, t1, t_eval) are always FP64.  The state dtype (y0, y_eval,
 *    y_final, mu, A, gradients) follows tode_options.prec: double for
 *    TODE_F64, float for TODE_F32 and TODE_BF16W.
 *  - Layouts are row-major, instance-major: y0 [B][D], y_eval [B][K][D],
 *    t_eval [B][K], A [B][D][D].
 */
#ifndef TODE_H
#define TODE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TODE_VERSION 1

typedef enum {
  TODE_OK = 0,
  TODE_EINVAL = 1,        /* bad argument (null pointer, size, option) */
  TODE_EWORKSPACE = 2,    /* workspace / tape / scratch too small or misaligned */
  TODE_ECUDA = 3,         /* a CUDA runtime call failed */
  TODE_EUNSUPPORTED = 4,  /* combination not built (field, D, precision) */
  TODE_ETIMEOUT = 5       /* a bounded host wait gave up */
} tode_err;

typedef enum { TODE_VDP = 1, TODE_LINEAR = 2, TODE_MLP = 3 } tode_field_kind;

/* TODE_F64: FP64 state and arithmetic.  TODE_F32: FP32 state (compensated
 * summation of the state updates), FP64 time.  TODE_BF16W (MLP only): BF16
 * weights on tensor cores, FP32 accumulation, FP32 state, FP64 time; the
 * field's input [y; t] enters as two BF16 terms (hi + lo), hidden
 * activations are rounded to BF16.  TODE_BF16W_SPLIT: as TODE_BF16W but the
 * hidden activations are also carried as two BF16 terms (twice the tensor
 * work, ~16 significant bits instead of 8). */
typedef enum { TODE_F64 = 0, TODE_F32 = 1, TODE_BF16W = 2, TODE_BF16W_SPLIT = 3 } tode_prec;

/* TODE_PLAIN: one kernel launch per step over the whole masked batch.
 * TODE_FUSED: one persistent launch; every worker integrates its instance to
 * the end and then takes the next one (work stealing). */
typedef enum { TODE_PLAIN = 0, TODE_FUSED = 1 } tode_form;

/* Per-instance status[] values. */
enum {
  TODE_S_SUCCESS = 0,       /* reached t1 */
  TODE_S_MAX_STEPS = 1,     /* max_steps attempted steps without reaching t1 */
  TODE_S_DT_UNDERFLOW = 2,  /* step size underflowed with finite errors */
  TODE_S_NONFINITE = 3,     /* step size underflowed while the state was non-finite */
  TODE_S_INVALID_INPUT = 4  /* t0/t1/t_eval not finite, t_eval not ordered from t0 towards t1
                               or outside the range */
};

/* The vector field f(t, y) (built-in kinds only).
 *  TODE_VDP:    Van der Pol, Eq. 1 as a first-order system, D = 2:
 *               f = (y2, mu_i (1 - y1^2) y2 - y1).  mu: [B] state dtype.
 *  TODE_LINEAR: f = A_i y.  A: [B][D][D] state dtype; D in {1,2,4,8,16,32}.
 *  TODE_MLP:    f = W_L tanh(... tanh(W_1 [y; t] + b_1) ...) + b_L.
 *               n_layers weight matrices, widths (host) [n_layers+1] with
 *               widths[0] = D + 1 and widths[n_layers] = D; W (host array of
 *               device pointers) W[l] is [widths[l+1]][widths[l]] BF16
 *               (uint16 bit patterns); b (host array of device pointers)
 *               b[l] is [widths[l+1]] float (NULL = zero).  Built shapes:
 *               widths {33, 128, 128, 32} and {65, 512, 512, 512, 64};
 *               both forms. */
typedef struct {
  tode_field_kind kind;
  int B;
  int D;
  const void* mu;
  const void* A;
  int n_layers;
  const int* widths;
  const void* const* W;
  const float* const* b;
} tode_field_desc;

typedef struct {
  double rtol, atol;          /* scalar tolerances */
  const double* rtol_b;       /* optional per-instance tolerances [B] (device), NULL = scalar */
  const double* atol_b;
  /* controller: factor = safety * err^-beta1 * err_prev^beta2 *
   * err_prev2^-beta3 (beta3 below), clamped to [fac_min, fac_max]; beta2 =
   * beta3 = 0 is the integral controller of App. A. */
  double safety, fac_min, fac_max, beta1, beta2;
  double h0;                  /* > 0: first step size; 0: starting-step heuristic */
  int max_steps;              /* attempted steps per instance (>= 1) */
  tode_prec prec;
  tode_form form;
  /* launch tuning (0 = default / autotuned) */
  int group;                  /* lanes per instance (linear field, D = 16: 4, 8 or 16) */
  int block;                  /* threads per block (multiple of 32, <= 256; 0 = 128, or
                                 fewer when the batch has under 128 threads per SM);
                                 Van der Pol and linear: tode_solve and tode_adjoint */
  int ctas_per_sm;            /* fused form: resident CTAs per SM; MLP field, wide
                                 network: tode_adjoint's slices of instances as
                                 a multiple (1..4, 0 = 1) of one CTA per SM */
  int poll_every;             /* plain form: steps between host polls */
  /* work order of the solvers (both forms, every field): 0 = index order,
   * 1 = longest integration interval |t1 - t0| first (lane groups that
   * share a warp then tend to take similar step counts, and long instances
   * start early so the persistent grid's tail shortens; a warp's
   * per-instance stores scatter).  Results do not depend on it; the
   * autotuner tries both. */
  int order;
  /* 0 = every instance solved independently (Sec. 3).  1 = joint
   * ("stacked") solving, the semantics Sec. 4.1 compares against: the batch
   * is one problem of size B*D with one step size, one RMS error norm over
   * all B*D components and one accept/reject decision per attempt.  Van der
   * Pol and linear fields, scalar rtol/atol; every instance must have the
   * same t0, t1 and t_eval as instance 0, else every instance is reported
   * TODE_S_INVALID_INPUT.  n_acc/n_rej/status are the problem's, repeated
   * for every instance.  One launch per attempt (form and order do not
   * apply; block, ctas_per_sm and poll_every do); a tape must be
   * stride 1 with h_acc, and tode_adjoint then reverses the shared mesh
   * per instance as usual. */
  int joint;
  /* derivative term of the PID controller (App. C: the decision looks at
   * the last three error estimates): the exponent of err_prev2, the error
   * of the accepted step before the previous one (1 before there is one).
   * 0 = the PI / I controller.  A strided tape needs err_prev2 when it is
   * not 0. */
  double beta3;
  /* the Runge-Kutta pair: TODE_DOPRI5 (0, Dormand & Prince 1980, the
   * paper's method throughout) or TODE_TSIT5 (1, Tsitouras 2011, which App.
   * A names as also available); both are 5(4) pairs with FSAL and an order-4
   * dense output, swapped by tableau only.  tsit5 covers every field (the
   * MLP field with prec TODE_BF16W_SPLIT), joint solving and the joint
   * continuous adjoint: tode_solve, tode_adjoint, tode_t_bounds_grad and
   * tode_joint_adjoint; the MLP field's TODE_BF16W form returns
   * TODE_EUNSUPPORTED with it. */
  int method;
} tode_options;

enum { TODE_DOPRI5 = 0, TODE_TSIT5 = 1 };

/* Checkpoint tape written by tode_solve for tode_adjoint.  Slot j of
 * instance i holds the solver state at the start of accepted step j*stride
 * (state y, its FSAL stage k1, time t, proposed step h, previous error,
 * flags), from which tode_adjoint re-runs the forward bit for bit.
 * Instance i needs ceil(n_acc[i] / stride) slots; tode_solve never writes
 * past `slots`, and tode_adjoint reports instances that needed more through
 * its `overflow` output.
 * With stride 1 and h_acc given (the same tape struct for both calls), every
 * accepted step is on the tape with its size and tode_adjoint reverses it
 * directly, without re-running the forward's attempts.
 * MLP field: the adjoint reverses every step from its recorded stage
 * inputs, so it takes a stride-1 tape with y, t, h_acc and y_stage; a solve
 * given a tape with stride > 1 records checkpoints for tode_mlp_resolve
 * instead (y, y_lo, k1, t, h, err_prev, flags and, when beta3 != 0,
 * err_prev2).
 * Every array is instance-major ([B][slots]...): the slots of one instance
 * are contiguous, so a lane group's successive checkpoint stores (and the
 * adjoint's loads) stay within the same cache lines.  Every array must be
 * 16-byte aligned (TODE_EINVAL otherwise).
 * A stride-1 tape with h_acc needs only y, t, h_acc and either k1 or
 * y_stage: y_lo, h, err_prev and flags (and k1 when y_stage is given) may
 * be NULL and are then not written -- they serve the re-run of strided
 * segments only.  The MLP field never needs k1. */
typedef struct {
  int slots;
  int stride;
  void* y;          /* [B][slots][D] state dtype */
  void* y_lo;       /* [B][slots][D] float: compensation term of an FP32 state
                       (TODE_F32 / TODE_BF16W); ignored for TODE_F64 (may be NULL) */
  void* k1;         /* [B][slots][D] state dtype: f(t, y) carried by FSAL */
  double* t;        /* [B][slots] */
  void* h;          /* [B][slots] state dtype: step proposed for the next attempt */
  void* err_prev;   /* [B][slots] state dtype */
  int32_t* flags;   /* [B][slots] */
  void* h_acc;      /* [B][slots] state dtype: size of the accepted step that
                       starts at the slot (written when that step is accepted;
                       required for the MLP field, optional otherwise) */
  void* y_stage;    /* [B][slots][6][D] state dtype: the stage inputs Y_2..Y_7
                       of the accepted step (MLP field: required; other fields:
                       optional -- with stride 1 and h_acc the adjoint then
                       reads them instead of re-evaluating the stages) */
  void* err_prev2;  /* [B][slots] state dtype: the PID controller's second error
                       history entry; needed by a re-run tape when beta3 != 0,
                       may be NULL otherwise */
} tode_tape;

/* Per-attempt trace (testing and diagnostics): for instance i, attempt n <
 * cap: step start t, step size h, error norm err, accepted flag; len[i] =
 * min(attempts, cap).  All [B][cap] except len [B]. */
typedef struct {
  int cap;
  double* t;
  double* h;
  double* err;
  int32_t* accepted;
  int32_t* len;
} tode_trace;

/* Fills *o with the defaults: rtol = atol = 1e-6, safety 0.9, fac_min 0.2,
 * fac_max 10, beta1 0.2, beta2 = beta3 = 0 (integral controller), h0 = 0 (heuristic),
 * max_steps 100000, TODE_F32, TODE_FUSED, tuning fields 0, order 0, joint 0,
 * TODE_DOPRI5. */
void tode_default_options(tode_options* o);

/* Bytes of device workspace tode_solve needs for this problem (the base
 * pointer must be 256-byte aligned): for the Van der Pol and linear fields
 * a work counter, the work order (one int32 per instance) and, above 2048
 * instances, the work-order sort's per-CTA counts, plus the per-instance
 * solver state between launches for the plain form, or for joint solving a
 * control block, per-CTA partial sums and a double buffer of the state
 * (6 * B * D values: y, its FP32 compensation term, k1).
 * Returns 0 for an unsupported or invalid combination. */
size_t tode_workspace_size(const tode_field_desc* f, const tode_options* o, int K);

/* Solve all B instances (Sec. 3: independent parallel solving).
 *  y0 [B][D], t0 [B], t1 [B], t_eval [B][K] (K >= 0; NULL when K == 0).
 *  An instance with t1 < t0 (every field; the MLP field's time input is the
 *  caller's t) integrates backward in time with negative steps: its t_eval
 *  runs from t0 down to t1, its trace holds negative h, and its tape holds
 *  -t (the solver works in tau = -t with positive steps and the field -f;
 *  tode_adjoint reads it that way).
 *  Outputs: y_eval [B][K][D] (NULL when K == 0), y_final [B][D] (state at
 *  the last accepted step), n_acc, n_rej, n_feval, status [B] int32.
 *  Evaluation points not reached (failed instance) are NaN; instances with
 *  TODE_S_INVALID_INPUT get NaN outputs and zero counters.
 *  tape: NULL or a checkpoint tape to fill for tode_adjoint.
 *  yp_eval: NULL or [B][K][D] state dtype: dy/dt at every evaluation point,
 *  the derivative of the dense-output interpolant there (f(t0, y0) at points
 *  equal to t0; NaN where y_eval is NaN).  Every field, independent solving
 *  (TODE_EUNSUPPORTED for a joint solve); for the MLP field the derivative
 *  is formed from the tensor-core stage values k_i in FP32, and an instance
 *  with t1 = t0 and points spends one evaluation round on f(t0, y0) (its
 *  counters stay 0).  With it, the gradient
 *  of a loss with respect to t_eval is <dL/dy_eval, yp_eval> per point
 *  (tode_t_eval_grad).
 *  trace: NULL or a per-attempt trace to fill.
 *  workspace: >= tode_workspace_size bytes, 256-byte aligned. */
tode_err tode_solve(const tode_field_desc* f, const tode_options* o, const void* y0,
                    const double* t0, const double* t1, const double* t_eval, int K,
                    void* y_eval, void* yp_eval, void* y_final, int32_t* n_acc, int32_t* n_rej,
                    int32_t* n_feval, int32_t* status, const tode_tape* tape,
                    const tode_trace* trace, void* workspace, size_t ws_bytes, void* stream);

/* Re-solve one checkpointed segment of an MLP-field solve (the budgeted
 * adjoint of App. A's backpropagation through the solver: the stages are
 * recomputed from checkpointed step-start states and step sizes).  A
 * tode_solve of the MLP field given a tape with stride m > 1 writes no stage
 * inputs; it records, at the start of every m-th accepted step, the whole
 * solver state (y, y_lo, k1, t, h = the step proposed for the first attempt,
 * err_prev, err_prev2 when beta3 != 0, flags).  This call runs, for every
 * instance, the accepted steps seg*m .. seg*m + m - 1 of that solve again from
 * checkpoint slot seg -- bit for bit the same attempts -- and fills seg_tape
 * (stride 1, slots >= m, h_acc and y_stage) with them, writing nothing else
 * of the solve.  Outputs per instance: seg_n [B] int32, the segment's accepted
 * steps (0 past the instance's last step); seg_t0, seg_t1 [B] double, its
 * bounds in the caller's time (both t1 when seg_n = 0).  tode_adjoint with t0
 * = seg_t0, t1 = seg_t1, n_acc = seg_n, the forward's status, seg_tape,
 * gy_final = the cotangent at seg_t1 and gy_eval zero outside (seg_t0,
 * seg_t1] (for seg > 0; [t0, seg_t1] for seg 0) reverses the segment and
 * returns the cotangent at seg_t0 in gy0.  n_acc: the solve's accepted-step
 * counts.  The fused form, prec TODE_BF16W_SPLIT (TODE_EUNSUPPORTED
 * otherwise); workspace as for tode_solve with K = 0.  Enqueued on stream;
 * allocates nothing. */
tode_err tode_mlp_resolve(const tode_field_desc* f, const tode_options* o, const double* t0,
                          const double* t1, const int32_t* n_acc, const tode_tape* ckpt, int seg,
                          const tode_tape* seg_tape, int32_t* seg_n, double* seg_t0,
                          double* seg_t1, void* workspace, size_t ws_bytes, void* stream);

/* Bytes of device scratch tode_adjoint needs (256-byte aligned base).  For
 * the MLP field it depends on the current device's SM count and, for the
 * wide network, on tape->slots: its reverse rounds stage the layer inputs
 * and cotangents of every (instance, step, stage) for the weight-gradient
 * products, one batch slice of SMs x 64 instances at a time, 7 * slots
 * rounds of 64 rows per SM (about 0.8 MB per round; gigabytes for a few
 * thousand-step slices). */
size_t tode_adjoint_scratch_size(const tode_field_desc* f, const tode_options* o,
                                 const tode_tape* tape);

/* Discrete adjoint of the fixed-mesh map of a previous tode_solve with the
 * same f, o, inputs and a filled tape (App. A: gradients by backpropagation
 * through the solver).  The mesh (accepted t_n, h_n) is a constant.  For
 * every instance it reverses the accepted steps -- from the recorded stage
 * inputs when the tape has them (y_stage; required for the MLP field),
 * otherwise recomputing the stages from the checkpoints -- and writes
 *   gy0 [B][D]       = dL/dy0
 *   gparam           = VDP: dL/dmu [B]; LINEAR: dL/dA [B][D][D] (state
 *                      dtype, per instance); MLP: NULL, or [B] double that
 *                      receives each instance's time-translation sum S_t,
 *                      the sum over its reversed stages of the cotangent of
 *                      the network's time input = dL/d(delta) when t0, t1
 *                      and the instance's evaluation points all move by
 *                      delta (NaN where the gradients are NaN); the input
 *                      tode_t_bounds_grad takes for dL/dt0 of this field
 *   gW, gb           = MLP only (host arrays of device pointers): dL/dW_l
 *                      [widths[l+1]][widths[l]] and dL/db_l [widths[l+1]],
 *                      float, summed over the batch in a fixed order
 *                      (deterministic); overwritten, not accumulated
 * from gy_eval [B][K][D] = dL/dy_eval (NULL = 0) and gy_final [B][D] =
 * dL/dy_final (NULL = 0).  n_acc and status are the forward's outputs;
 * instances whose status is not TODE_S_SUCCESS get NaN gradients.
 * overflow (int32, device) is set to 1 when some instance needed more tape
 * slots than the forward had (that instance's gradients are NaN). */
tode_err tode_adjoint(const tode_field_desc* f, const tode_options* o, const double* t0,
                      const double* t1, const double* t_eval, int K, const int32_t* n_acc,
                      const int32_t* status, const tode_tape* tape, const void* gy_eval,
                      const void* gy_final, void* gy0, void* gparam, float* const* gW,
                      float* const* gb, int32_t* overflow, void* scratch, size_t scratch_bytes,
                      void* stream);

/* Size of the device scratch that tode_adjoint_static keeps inside the
 * library (32 MiB on every GPU that loads it). */
#define TODE_STATIC_ADJOINT_SCRATCH_BYTES (32u << 20)

/* tode_adjoint without a scratch argument, for callers that cannot allocate
 * device memory: code that only receives its input and output buffers from a
 * host framework (a plugin interface, for instance) and has no allocator of
 * its own, or code that must not call cudaMalloc in a latency-critical loop
 * because it can synchronise the device.  The paper has no counterpart; this
 * is a deployment convenience.
 *  - Arguments, outputs and errors are those of tode_adjoint minus scratch,
 *    checked in the same order (an invalid argument or tape is
 *    TODE_EINVAL / TODE_EUNSUPPORTED whatever its size).  The scratch is a
 *    library-owned device array of TODE_STATIC_ADJOINT_SCRATCH_BYTES; a
 *    valid problem whose tode_adjoint_scratch_size exceeds it is rejected
 *    with TODE_EWORKSPACE before any device work (a strided tape: lower
 *    tape->stride; otherwise split the batch).  The wide MLP network
 *    (D = 64, hidden 512) stages gigabytes of layer rows for its weight
 *    gradients and is always rejected this way; the D = 32, hidden 128
 *    network fits.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *  - The first call on each device looks up the array's device address with
 *    that device current (cudaGetSymbolAddress) and caches it; make that
 *    first call before any stream capture.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents (the work counter is cleared on `stream` at every call).  Calls
 *    that can overlap on the GPU (different streams, or several host
 *    threads) race on it: serialise them. */
tode_err tode_adjoint_static(const tode_field_desc* f, const tode_options* o, const double* t0,
                             const double* t1, const double* t_eval, int K, const int32_t* n_acc,
                             const int32_t* status, const tode_tape* tape, const void* gy_eval,
                             const void* gy_final, void* gy0, void* gparam, float* const* gW,
                             float* const* gb, int32_t* overflow, void* stream);

/* Gradient with respect to the evaluation times of a solve that wrote
 * yp_eval: g_t_eval[i][q] = sum_j gy_eval[i][q][j] yp_eval[i][q][j] (the
 * output y(t_eval[i][q]) moves with its time at the rate yp_eval).  gy_eval
 * and yp_eval [B][K][D] in the state dtype (prec TODE_F64 or TODE_F32),
 * g_t_eval [B][K] double, all device pointers; enqueued on stream. */
tode_err tode_t_eval_grad(int B, int K, int D, tode_prec prec, const void* gy_eval,
                          const void* yp_eval, double* g_t_eval, void* stream);

/* Gradients with respect to the integration bounds t0 and t1 of a solve's
 * frozen map (the discrete-adjoint reading of App. A, extended to the two
 * boundary times): every accepted step size but the last and every
 * evaluation point's step are held, t0 moves every mesh point before t1, and
 * the last step h = t1 - t_{N-1} absorbs the change.  Every field solved
 * independently (TODE_EUNSUPPORTED for a joint solve; the MLP field with
 * prec TODE_BF16W_SPLIT), a stride-1 tape with h_acc filled by the solve
 * (TODE_EINVAL for a strided tape).
 *  g_t1 [B] (double, required) = dL/dt1: the last step size's cotangent
 *  (for the MLP field, whose stage times t_n + c_i h move with h, through
 *  its time input too; that step is re-run in FP32 on the CUDA cores).
 *  g_t0 [B] (double, may be NULL) = dL/dt0 = S_t - sum_q <gy_eval[q],
 *  yp_eval[q]> - dL/dt1: translating both bounds and every point by delta
 *  changes L by S_t delta, S_t = 0 for the autonomous Van der Pol and linear
 *  fields; for the MLP field g_t0 must hold S_t on entry (tode_adjoint's
 *  gparam of the same cotangents) and is overwritten.  Needs yp_eval
 *  [B][K][D] from the same solve (tode_solve's dy/dt output) when gy_eval is
 *  given.
 * gy_eval [B][K][D] and gy_final [B][D] (state dtype, NULL = 0) as for
 * tode_adjoint; instances whose status is not TODE_S_SUCCESS (or that needed
 * more tape slots than the tape has) get NaN; an instance with t1 = t0 gets
 * g_t1 = 0.  Backward instances (t1 < t0) are handled in their own
 * direction.  Enqueued on stream; allocates nothing. */
tode_err tode_t_bounds_grad(const tode_field_desc* f, const tode_options* o, const double* t0,
                            const double* t1, const double* t_eval, int K, const int32_t* n_acc,
                            const int32_t* status, const tode_tape* tape, const void* gy_eval,
                            const void* gy_final, const void* yp_eval, double* g_t0,
                            double* g_t1, void* stream);

/* Joint continuous adjoint (App. A, the CNF benchmark's "torchode-joint"
 * backward pass): the adjoint equation of the whole batch solved as ONE
 * problem of size 2BD + P -- the state integrated back from y(t1), its
 * adjoint a and the adjoint of the P shared network parameters,
 *   dy/dt = f(t, y_b),  da_b/dt = -J_f(t, y_b)^T a_b,
 *   dabar/dt = -sum_b (df/dtheta)(t, y_b)^T a_b,
 * integrated backward from t1 to t0 by dopri5 with one step size, one RMS
 * error norm over all 2BD + P components (scale atol + rtol max(|z|,
 * |z1|)) and one accept/reject decision, the controller of tode_options and
 * the starting-step heuristic with its norms over the whole system.  The
 * integration stops at every evaluation point strictly inside (t0, t1) and
 * adds that point's cotangent to a (the loss jumps there); points at t1
 * start a, points at t0 add at the end.  The MLP field of the D = 32, H =
 * 128 network (TODE_EUNSUPPORTED otherwise), prec TODE_BF16W_SPLIT, scalar
 * tolerances, either pair; t0 < t1 shared by the batch (host doubles),
 * t_eval [K] host, shared, ordered from t0 to t1.
 *   y1 [B][D] float (device): y(t1) from the forward solve.
 *   gy_eval [B][K][D], gy_final [B][D] (device float, NULL = 0).
 *   gy0 [B][D] (device float, written): dL/dy0 = a(t0).
 *   gW[l], gb[l] (device float, written): dL/dtheta = abar(t0), shaped like
 *     the field's W[l] ([out][in]) and b[l].
 *   y0 [B][D] (device float, written; may be NULL): y integrated back to t0.
 *   stats (host int32 [4], written): accepted and rejected steps and
 *     augmented evaluations over all segments, and the status
 *     (TODE_S_SUCCESS or the first failure).
 * workspace: tode_joint_adjoint_workspace_size bytes, 256-byte aligned.
 * Synchronous: the host reads the decision every few attempts; enqueued on
 * stream, returns when the result is there.  TODE_ETIMEOUT if a tensor-core
 * wait gave up. */
size_t tode_joint_adjoint_workspace_size(const tode_field_desc* f, const tode_options* o);
tode_err tode_joint_adjoint(const tode_field_desc* f, const tode_options* o, double t0, double t1,
                            const double* t_eval, int K, const void* y1, const void* gy_eval,
                            const void* gy_final, void* gy0, float* const* gW, float* const* gb,
                            void* y0, int32_t* stats, void* workspace, size_t ws_bytes,
                            void* stream);

/* The MLP field's tensor-core building block on its own, for checking the
 * operand layouts and tensor-memory conventions against a plain product:
 * C[M][N] = sum_k A(m,k) B(n,k) with A, B BF16 (uint16 bit patterns) and C
 * float row-major, on one CTA with tcgen05.mma and FP32 accumulation in
 * tensor memory.  A is [M][K] row-major (K-major operand) or, with flags bit
 * 0, [K][M] row-major (MN-major operand); likewise B is [N][K] or, with bit
 * 1, [K][N].  Bit 2 swaps the two stride fields of MN-major descriptors.
 * M = 128 or 64; N, K multiples of 16 in [16, 256] (K <= 128 and N <= 144
 * when any flag is set; no MN-major A with M = 64).  With M = 64, C must hold
 * [128][N]: it receives all 128 tensor-memory lanes, each lane's N columns,
 * with -12345 wherever the MMA wrote nothing (this shows the M = 64
 * accumulator layout); with flags bit 3 (M = 64, N >= 48) each thread of
 * warp w instead writes the 16 values of one 16x32bx2 tensor-memory load
 * (half-split offset 32 columns) to C[32w + lane][0:16].  err (device int32)
 * is set to
 * 1 if the tensor cores did not signal completion within about a second (C
 * is then left unwritten). */
tode_err tode_tc_gemm(const void* A, const void* B, float* C, int M, int N, int K, int flags,
                      int32_t* err, void* stream);

/* Micro-benchmark kernels for the rooflines' denominators on the running
 * GPU (no paper counterpart: measurement infrastructure).  kind selects the
 * kernel: each thread of the grid x block launch runs iters iterations of 8
 * independent chains of one operation --
 *   TODE_PEAK_FMA32  FP32 fused multiply-add (2 FLOP each)
 *   TODE_PEAK_FFMA2  paired FP32 FMA, two lanes per instruction (4 FLOP)
 *   TODE_PEAK_FMA64  FP64 fused multiply-add (2 FLOP)
 *   TODE_PEAK_EX2    ex2.approx (one MUFU operation)
 *   TODE_PEAK_TANH   tanh.approx (one MUFU operation)
 * -- so one launch performs grid * block * iters * 8 operations;
 * TODE_PEAK_EMPTY launches an empty kernel (launch and graph-replay rates;
 * sink may be NULL).  sink (device, >= block floats) receives nothing in
 * practice: it only keeps the chains alive.  The caller times the launch
 * on `stream`.  TODE_EINVAL for a bad kind or shape. */
enum {
  TODE_PEAK_FMA32 = 0,
  TODE_PEAK_FFMA2 = 1,
  TODE_PEAK_FMA64 = 2,
  TODE_PEAK_EX2 = 3,
  TODE_PEAK_TANH = 4,
  TODE_PEAK_EMPTY = 5
};
tode_err tode_peak_kernel(int kind, int grid, int block, int iters, float* sink, void* stream);

/* Static text for an error code. */
const char* tode_strerror(tode_err e);

/* TODE_VERSION of the loaded library. */
int tode_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TODE_H */
