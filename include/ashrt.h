/*
 * ashrt.h -- C ABI of the GB300 (sm_103a) Stolt-based apex-shifted hyperbolic
 * Radon transform (ASHRT), its asymptote-shifted extension (AASHRT), and the
 * robust IRLS deblending solve built on them.
 *
 * Method: Ibrahim (2015), "Separating simultaneous seismic sources using
 * robust inversion of Radon and migration operators" (arxiv 1711.10214).
 *   ch. 5, Eqs ch5_forward_operator / ch5_adj_operator: L = S F^-1 M F,
 *          L^T = F^-1 M^T F S^T (Stolt map M, sum S over velocities);
 *   ch. 6, Eqs ch6_forward_operator / ch6_adj_operator: adds the asymptote
 *          time shift T = exp(-i w tau0), the sum A over (v, tau0) and the
 *          trace-sampling operator S;
 *   ch. 4, Eqs ch4_cost_fn, equ:10, equ:11, ch4_epcilon_r: robust l_p-l_q
 *          inversion by IRLS with an inner conjugate-gradient (CGLS) solve.
 *
 * Conventions shared by every call
 *   - Data (a common-receiver gather) is float32 [batch][nx][nt], t fastest.
 *   - Model is float32 [batch][nt0][nv][nx][nt]: one (tau, x_apex) panel per
 *     (asymptote shift tau0_j, velocity v_i), t (= tau) fastest.  Apex
 *     positions equal trace positions (x_a == x, ch. 6).
 *   - All array arguments named *_dev are device pointers owned by the
 *     caller, contiguous, 4-byte aligned; nothing here frees them.
 *   - Every call is asynchronous on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream) unless documented otherwise.  Calls never
 *     allocate device memory except ashrt_plan_create.
 *   - Functions return an ashrt_status; no exception crosses the ABI.  The
 *     text of the last error of the calling thread is ashrt_last_error().
 *   - A plan may be used from one thread at a time: forward, adjoint and the
 *     deblend solve all use the plan's workspace.
 */
#ifndef ASHRT_H
#define ASHRT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ASHRT_OK = 0,
  ASHRT_EINVAL = 1,     /* invalid argument (sizes, NULL pointers, grids) */
  ASHRT_ENOMEM = 2,     /* device allocation failed at plan creation */
  ASHRT_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  ASHRT_ENAN = 4,       /* non-finite value in the input data */
  ASHRT_ENOTCONV = 5,   /* IRLS stopped without meeting its tolerance (informative) */
  ASHRT_ETIMEOUT = 6,   /* a device-side bounded wait ran out */
  ASHRT_EINTERNAL = 7   /* internal consistency check failed */
} ashrt_status;

typedef struct ashrt_plan ashrt_plan;

/* Operator options (ch. 5 "zero padding"; ch. 4 wavelet C; ch. 5 band limit). */
typedef struct {
  int pad_t;              /* Nt = next power of two >= pad_t * nt (default 2), at least 64 */
  int pad_x;              /* Nx = next power of two >= pad_x * nx (default 2), at least 16 */
  float fmax_hz;          /* > 0: zero |f| > fmax in both directions; 0 = none */
  float wavelet_peak_hz;  /* > 0: apply the zero-phase Ricker amplitude spectrum
                             W(f) = (f/fp)^2 exp(1 - (f/fp)^2) as C (forward) and
                             C^T (adjoint); 0 = off */
  int max_batch;          /* largest batch any call will pass (workspace size) */
  int with_solver;        /* 1: also allocate the IRLS/CGLS vectors */
} ashrt_opts;

/* Fills *opts with the defaults: pad 2/2, no band limit, no wavelet,
 * max_batch 1, with_solver 0. */
void ashrt_default_opts(ashrt_opts* opts);

/*
 * Creates a plan on the current CUDA device.
 *   nt, nx        samples per trace and traces per gather (nt >= 2, nx >= 2,
 *                 Nt <= 4096, Nx <= 2048 after padding)
 *   dt, dx        sample interval [s] and trace spacing [m]
 *   velocities    host array of nv > 0 scan velocities [m/s] (>= 0)
 *   apex_x        host array of napex apex positions [m]; must be NULL or the
 *                 trace positions j*dx (napex == nx): the Stolt operator
 *                 requires x_a == x (ch. 6)
 *   t0_shifts     host array of nt0 asymptote shifts tau0 [s], or NULL with
 *                 nt0 = 1 for plain ASHRT (tau0 = 0, ch. 6: AASHRT reduces to
 *                 ASHRT at zero shift)
 *   opts          may be NULL (defaults)
 * The cone membership of every (w, k_x) bin is decided on the host in IEEE
 * double as k*k > a*a with a = ((v*|l|)*Nt)*dt/(Nx*dx) (bin units).
 * Allocates all device tables and workspace; returns ASHRT_ENOMEM if that
 * fails.  *out receives the plan (NULL on failure).
 */
ashrt_status ashrt_plan_create(ashrt_plan** out, int nt, int nx, double dt, double dx,
                               const float* velocities, int nv,
                               const float* apex_x, int napex,
                               const float* t0_shifts, int nt0,
                               const ashrt_opts* opts);

/*
 * Creates a plan whose data traces lie at arbitrary positions (ch. 6: for
 * irregular spatial sampling the trace-axis Fourier operator F is replaced by
 * a discrete Fourier transform evaluated at the trace positions).  The model
 * keeps the regular apex grid x_a = j dx, j < nx (the Stolt map needs it);
 * the data of every call on this plan is [batch][nr][nt], trace j recorded at
 * trace_x[j] metres (host array, any finite values, in any order), and trace
 * masks are [batch][nr].  The forward synthesises each trace from the half
 * spectrum of the padded apex axis,
 *   d_j(t) = sum_{l=0}^{Nx/2} c_l Re( exp(+2 pi i l x_j / (Nx dx)) Y_l(t) ),
 * c_0 = c_{Nx/2} = 1, c_l = 2 otherwise (the Nyquist term enters as
 * cos(pi x_j / dx)), and the adjoint is its exact transpose; with trace_x[j]
 * = j dx and nr = nx this is the plan of ashrt_plan_create.  Every other
 * argument as ashrt_plan_create (apex positions are j dx); max_batch <= 65535.
 * The data-side transforms are dense contractions costing about
 * 4 nr nt (Nx/2 + 1) flops per gather and direction.  ashrt_forward,
 * ashrt_adjoint, robust_irls_deblend and ashrt_fista accept the plan; the
 * batch layer (ashrt_batch_*) and ashrt_forward_static do not take
 * irregular traces.
 */
ashrt_status ashrt_plan_create_irregular(ashrt_plan** out, int nt, int nx, double dt, double dx,
                                         const float* velocities, int nv,
                                         const float* t0_shifts, int nt0,
                                         const double* trace_x, int nr,
                                         const ashrt_opts* opts);

/* Frees a plan and its device memory (synchronises the device first). NULL is a no-op. */
void ashrt_plan_destroy(ashrt_plan* plan);

/* Reports padded sizes, panel count P = nv*nt0 and the workspace held. Any out pointer may be NULL. */
ashrt_status ashrt_plan_info(const ashrt_plan* plan, int* Nt, int* Nx, int* n_panels,
                             size_t* workspace_bytes);

/*
 * Forward (demigration / modelling), ch. 5 Eq. ch5_forward_operator and
 * ch. 6 Eq. ch6_forward_operator:
 *   d = S C F^-1 sum_{tau0} T(tau0) sum_v M_v F m,   T = exp(-i w tau0).
 *   m_dev           [batch][nt0][nv][nx][nt] float32 model (read)
 *   d_dev           [batch][nx][nt] float32 data (written)
 *   trace_mask_dev  [batch][nx] float32 sampling weights S (1 keep, 0 drop) or NULL
 * batch must be in [1, max_batch].  Uses the plan workspace.
 */
ashrt_status ashrt_forward(const ashrt_plan* plan, const float* m_dev, float* d_dev,
                           const float* trace_mask_dev, int batch, void* stream);

/*
 * Adjoint (migration), ch. 5 Eq. ch5_adj_operator and ch. 6 Eq.
 * ch6_adj_operator: the exact transpose of ashrt_forward (linear-interpolation
 * weights transposed, conjugate phase), so <L m, d> = <m, L^T d> to rounding.
 *   d_dev  [batch][nx][nt] (read);  m_dev [batch][nt0][nv][nx][nt] (written)
 */
ashrt_status ashrt_adjoint(const ashrt_plan* plan, const float* d_dev, float* m_dev,
                           const float* trace_mask_dev, int batch, void* stream);

/*
 * Forward operator without a plan and without any device allocation.  The
 * paper has no counterpart: this exists for callers that cannot allocate
 * device memory -- a host application that owns the GPU's memory through its
 * own allocator or a fixed budget and passes this library only its input and
 * output buffers, or a latency-critical loop in which a cudaMalloc would
 * synchronise the device.  Computes what ashrt_forward computes for a plan
 * with the same arguments: the same tables and kernels, with the row kernel
 * in its radix-8 form (a plan's variant 3; a plan's default for Nt 1024..4096
 * is the radix-16 forward, which agrees with it to rounding).
 *   nt, nx, dt, dx, velocities/nv, t0_shifts/nt0, opts: as ashrt_plan_create
 *     (apex positions are the trace positions; opts->max_batch and
 *     opts->with_solver are ignored)
 *   m_dev, d_dev, trace_mask_dev, batch, stream: as ashrt_forward
 * Scratch: all tables and the operator workspace live in one static device
 * array of 16 MiB that every GPU loading this library holds until the process
 * exits.  A call whose tables plus workspace exceed it (roughly batch * nv *
 * nt0 * (Nx/2 + 1) * nt * 8 bytes) returns ASHRT_EINVAL with the size it
 * needed.  The call allocates nothing: no cudaMalloc, no cudaFree.
 * Each call looks up that array's device address on the current device
 * (cudaGetSymbolAddress, with the caller's device current), so the entry
 * point follows cudaSetDevice and survives cudaDeviceReset.  Every call
 * rewrites the shared array: the tables are uploaded with cudaMemcpyAsync on
 * `stream` from host memory that lives only for the call, so the call is
 * refused (ASHRT_EINVAL) while `stream` -- or, for the legacy stream, any
 * stream of the device -- is being captured into a CUDA graph.  Calls that
 * overlap on the GPU -- on different streams, or from different threads --
 * race on the array: serialise them.
 */
ashrt_status ashrt_forward_static(int nt, int nx, double dt, double dx,
                                  const float* velocities, int nv,
                                  const float* t0_shifts, int nt0,
                                  const ashrt_opts* opts, const float* m_dev, float* d_dev,
                                  const float* trace_mask_dev, int batch, void* stream);

/*
 * Time-domain ASHRT / AASHRT by hyperbolic summation: the classical form of
 * the operator pair (ch. 3 Table ch3_table_Radon_operators, ASHRT row; ch. 6
 * Eq. ch6_AASHRT_adjoint) that ch. 5 compares the Stolt form against, with
 * cost O(nx^2 nt nv nt0) per gather.  The adjoint sums each trace x_r along
 * the hyperbola t = tau0 + sqrt(tau^2 + (x_r - x_a)^2 / v^2) of every
 * (tau, v, x_a, tau0), reading d at the fractional time by linear
 * interpolation between samples (a sample at or past nt reads 0); the
 * forward is its exact transpose.  No padding, no wavelet, no band limit:
 * this is a different discretisation of the operator than the Stolt pair,
 * not a copy of it.
 *   nt (2..4096), nx (>= 1), dt, dx (> 0)   gather sampling
 *   velocities   host array of nv scan velocities [m/s], each > 0
 *   t0_shifts    host array of nt0 asymptote shifts [s], each >= 0, or NULL
 *                with nt0 = 1 (ASHRT); nv * nt0 <= 256
 *   m_dev        [batch][nt0][nv][nx][nt] model (read by forward, written by adjoint)
 *   d_dev        [batch][nx][nt] data (written by forward, read by adjoint)
 * Asynchronous on `stream`, one kernel launch, no allocation, no plan.  The
 * forward accumulates with shared-memory atomic adds, so its last bits
 * depend on scheduling.  Argument errors return ASHRT_EINVAL before any
 * CUDA call.
 */
ashrt_status ashrt_td_forward(int nt, int nx, double dt, double dx, const float* velocities,
                              int nv, const float* t0_shifts, int nt0, const float* m_dev,
                              float* d_dev, int batch, void* stream);
ashrt_status ashrt_td_adjoint(int nt, int nx, double dt, double dx, const float* velocities,
                              int nv, const float* t0_shifts, int nt0, const float* d_dev,
                              float* m_dev, int batch, void* stream);

/* Options of the robust solve (ch. 4). */
typedef struct {
  double p;               /* misfit norm exponent, 0 < p <= 2 (1 = robust) */
  double q;               /* model norm exponent, 0 < q <= 2 (1 = sparse) */
  int n_outer;            /* IRLS (reweighting) iterations, <= 64 */
  int n_cg;               /* CGLS iterations per outer iteration */
  double tol;             /* stop a gather when |J_k - J_k-1| / J_k-1 < tol; 0 = never */
  double b_r;             /* eps_r = b_r MAD(r) / 0.6745 (default 1.345) */
  double b_m;             /* eps_m = b_m max|m| / 100 (default 1) */
  double mu;              /* trade-off of Eq. equ:11 (default 0: CG count regularises) */
  int warm_start_cg;      /* 1: start CGLS of outer k from u0 = W_m m_{k-1} (default 1) */
  double eps_r_fixed;     /* > 0: use this eps_r instead of the MAD rule */
  double eps_m_fixed;     /* > 0: use this eps_m instead of the max rule */
  const float* trace_mask_dev;  /* [batch][nx] sampling weights S, or NULL */
  const float* apex_mask_dev;   /* [batch][nx] 1 = apex position present, 0 = absent: the
                                   model panels of an absent apex are removed from the
                                   solve (W_m^-1 = 0 there, so that model column stays 0);
                                   NULL = all present.  Used to solve a narrower gather
                                   inside a wider one (uneven batches). */
  int use_graph;                /* 1: record the whole iteration sequence as a CUDA graph on
                                   the first call and replay it while the arguments repeat
                                   (ignored when tol > 0, which synchronises per iteration) */
  const float* m0_dev;          /* [batch][nt0][nv][nx][nt] initial model (warm start), or
                                   NULL (cold start: m = 0, W_m = I at the first iteration).
                                   With m0 the first iteration already reweights: W_m from
                                   m0 and, unless wr0 is given, W_r from d - C S L m0. */
  const float* wr0_dev;         /* [batch][nx][nt] residual weights W_r of the first
                                   iteration (e.g. a learned prediction), or NULL */
  float* wr_out_dev;            /* [batch][nx][nt] written at the end: the residual weights
                                   max(|r|, eps_r)^((p-2)/2) of the final residual (what the
                                   next outer iteration would use), or NULL */
} irls_opts;

/* Per-gather outcome of the robust solve. */
typedef struct {
  int outer_done;         /* outer iterations actually run for this gather */
  int applies_fwd;        /* forward operator applications spent on it */
  int applies_adj;        /* adjoint operator applications spent on it */
  int flags;              /* bit 0: stopped on tol; bit 1: breakdown (zero CG denominator) */
  double misfit[64];      /* J_k = sum |r_i|^p over live samples after outer k (FP64) */
} irls_report;

/* Fills *opts with p = q = 1, n_outer 5, n_cg 20, tol 0, b_r 1.345, b_m 1, mu 0, warm start on. */
void irls_default_opts(irls_opts* opts);

/*
 * Robust Radon deblending of `batch` gathers (ch. 4, Eqs ch4_cost_fn, equ:10,
 * equ:11): minimise ||d - C S L m||_p^p + mu ||m||_q^q by IRLS; each outer
 * iteration sets W_r, W_m from the residual and model (eps_r from the MAD,
 * eps_m from max|m|; W = I at the first), then runs CGLS on
 * A = W_r S C L W_m^-1 with u = W_m m.  CG scalars and all norms are
 * accumulated in FP64, per gather.
 *   d_dev     [batch][nx][nt] pseudo-deblended gathers (read)
 *   m_dev     [batch][nt0][nv][nx][nt] Radon models (written)
 *   drec_dev  [batch][nx][nt] recovered gathers C L m, no mask (written; may be NULL)
 *   per_gather  host array of `batch` reports (may be NULL)
 * Requires a plan created with with_solver = 1.  Synchronises `stream` once
 * at the end (and once per outer iteration when tol > 0).  Returns
 * ASHRT_ENAN if d holds a non-finite value (m and drec are then untouched).
 */
ashrt_status robust_irls_deblend(const ashrt_plan* plan, const float* d_dev, float* m_dev,
                                 float* drec_dev, int batch, const irls_opts* opts,
                                 irls_report* per_gather, void* stream);

/*
 * Sparse inversion by FISTA for AASHRT interpolation (ch. 6, "Sparse
 * inversion": Eq. cost_fn with p = 2, q = 1):
 *   minimise J(m) = ||S (d - L m)||_2^2 + mu ||m||_1
 * with L the plan's forward and S the trace mask, by the fast iterative
 * shrinkage-thresholding algorithm (Beck and Teboulle 2009) with step 1/Lf,
 * Lf = 2 lambda_max(L^T S^T S L) from n_power iterations of Rayleigh's power
 * method started at v0 (the caller's random draw, normalised here).  The model
 * starts at zero; every gather runs n_iter iterations with its own Lf.
 *   d_dev           [batch][nx][nt] data (read; traces with mask 0 are ignored)
 *   trace_mask_dev  [batch][nx] sampling weights S, or NULL (all traces)
 *   v0_dev          [batch][nt0][nv][nx][nt] power-method start (read)
 *   m_dev           [batch][nt0][nv][nx][nt] the sparse model (written)
 *   drec_dev        [batch][nx][nt] L m on every trace -- the interpolated
 *                   gather -- or NULL
 *   lipschitz       host array of batch Lf values (written), or NULL
 * Requires a plan created with with_solver = 1 (its solver vectors are the
 * workspace).  Asynchronous on `stream` until one synchronisation at the end.
 * lambda = 0 (nothing sampled) leaves that gather's model at zero.
 */
typedef struct {
  double mu;              /* trade-off of Eq. cost_fn, >= 0 (default 0) */
  int n_iter;             /* FISTA iterations, >= 1 (default 50) */
  int n_power;            /* power-method iterations, >= 1 (default 20) */
} fista_opts;
void fista_default_opts(fista_opts* opts);
ashrt_status ashrt_fista(const ashrt_plan* plan, const float* d_dev, const float* trace_mask_dev,
                         const float* v0_dev, float* m_dev, float* drec_dev, int batch,
                         const fista_opts* opts, double* lipschitz, void* stream);

/*
 * Acquisition model around the solve (ch. 2, Eqs ch2_blending and
 * pseudodeblending_equ).  A cube of common-shot gathers D [ns][nr][nt] is
 * blended into one continuous record per receiver b [nr][nb]; pseudo-
 * deblending cuts each shot's window back out (the exact transpose); sorting
 * swaps the two gather axes, [n0][n1][nt] -> [n1][n0][nt] (shot gathers to
 * the receiver gathers the solve works on, where the interference is
 * incoherent, and back).
 *   fire_dev   int32 device array [ns]: firing sample tau_i of shot i (any
 *              value; samples falling outside [0, nb) are dropped)
 *   blending        b[r, t'] = sum_i D[i, r, t' - tau_i]  (0 <= t' - tau_i < nt),
 *                   summed in shot order (no atomics: reproducible)
 *   pseudo-deblend  D[i, r, t] = b[r, tau_i + t]  (0 <= tau_i + t < nb, else 0)
 * Asynchronous on `stream`, one launch each, no allocation.  ns <= 8192 for
 * ashrt_blend; every other count <= 65535.  src and dst of the sort must not
 * overlap.
 */
ashrt_status ashrt_blend(const float* shots_dev, int ns, int nr, int nt, const int* fire_dev,
                         float* record_dev, int nb, void* stream);
ashrt_status ashrt_pseudo_deblend(const float* record_dev, int nr, int nb, const int* fire_dev,
                                  int ns, int nt, float* shots_dev, void* stream);
ashrt_status ashrt_sort_gathers(const float* src_dev, int n0, int n1, int nt, float* dst_dev,
                                void* stream);

/*
 * Autotuner (no counterpart in the paper): times forward+adjoint pairs of
 * `batch` gathers on the plan's sizes for each kernel variant -- the row
 * kernels' form (rows_minb 1, 2 or 3: radix-8 transforms with a register cap
 * for that many resident CTAs per SM, Nt 512..2048; for Nt 1024..4096 also
 * 4: radix-16 forward (three shared-memory passes per transform instead of
 * four) with the radix-8 adjoint, 5: radix-16 both, 6: radix-16 both with one
 * gather per CTA instead of an interleaved pair (half the shared memory, so
 * about twice the resident CTAs; per-bin tables read from L2 instead of
 * staged), 7: that forward with the radix-8 pair adjoint, 8: the radix-16
 * pair forward with that adjoint, 9: as 5 with the forward's per-bin sums in
 * tensor memory instead of registers (Nt = 2048 only, four CTAs per SM
 * instead of three; on other lengths the same kernels as 5); the default is 9
 * at Nt = 2048, 4 at Nt = 1024 and 4096, else 3)
 * and the trace-axis FFT column tile (16 or 8 columns for Nx <= 512) -- and
 * keeps the fastest in the plan; the plan's current choice is timed first and
 * another one replaces it only when it is more than 2% faster, so variants
 * within timing noise of each other do not flip from run to run.  With cache_path (a JSON-lines file, one object per
 * device and problem shape) a cached choice is reused without timing and new
 * choices are appended.  Allocates and frees temporary buffers; synchronises.
 * The chosen variants are returned in rows_minb / xfft_cols (may be NULL).
 * Every variant computes the same operator.
 */
ashrt_status ashrt_plan_autotune(ashrt_plan* plan, int batch, const char* cache_path,
                                 int* rows_minb, int* xfft_cols);
/* Sets the variants directly (rows_minb 1..9, xfft_cols 8 or 16); register
 * caps and column tiles that do not apply to the plan's sizes fall back to the
 * default kernel; rows_minb 4..9 on an Nt other than 1024, 2048 or 4096 is
 * ASHRT_EINVAL. */
ashrt_status ashrt_plan_set_variant(ashrt_plan* plan, int rows_minb, int xfft_cols);

/*
 * Batches of gathers with uneven trace counts (ashrt_batch_create: all with
 * the same nt; ashrt_batch_create_uneven below: uneven nt too).  The
 * gathers are independent (ch. 1: separation gather by gather is parallel
 * work); packed layouts concatenate them:
 *   data   : gather g is [nx_g][nt] at element offset nt * sum_{h<g} nx_h
 *   model  : gather g is [nt0][nv][nx_g][nt] at offset P nt sum_{h<g} nx_h
 * Gathers are grouped by padded width Nx (next power of two >= pad_x nx_g);
 * each class is solved as one batch of its widest gather's width, narrower
 * gathers padded with zero traces that are excluded from the solve (trace
 * mask for the data side, apex mask for the model side), which reproduces the
 * per-gather operator exactly.  opts->max_batch is the number of gathers of a
 * class resident on the device at once (default 64); larger classes are
 * processed in chunks.  Allocates at creation only.
 */
typedef struct ashrt_batch ashrt_batch;
ashrt_status ashrt_batch_create(ashrt_batch** out, int nt, const int* nx_per_gather, int ngather,
                                double dt, double dx, const float* velocities, int nv,
                                const float* t0_shifts, int nt0, const ashrt_opts* opts);
/* The same for gathers of uneven sample counts too: gather g is [nx_g][nt_g]
 * (model [nt0][nv][nx_g][nt_g]) at the packed offsets sum_{h<g} nx_h nt_h
 * (times P for the model); classes are formed per (nt, Nx). */
ashrt_status ashrt_batch_create_uneven(ashrt_batch** out, const int* nt_per_gather,
                                       const int* nx_per_gather, int ngather, double dt, double dx,
                                       const float* velocities, int nv, const float* t0_shifts,
                                       int nt0, const ashrt_opts* opts);
void ashrt_batch_destroy(ashrt_batch* batch);
/* Runs ashrt_plan_autotune on every class plan at the class's resident batch
 * (each (nt, Nx) class gets its own row-kernel variant and column tile);
 * cache_path as there.  Allocates temporary buffers and synchronises. */
ashrt_status ashrt_batch_autotune(ashrt_batch* batch, const char* cache_path);
/* Number of Nx classes, packed data / model element counts, device bytes held. */
ashrt_status ashrt_batch_info(const ashrt_batch* batch, int* n_classes, long long* data_elems,
                              long long* model_elems, size_t* workspace_bytes);
/* Forward / adjoint of every gather (packed layouts above), async on stream. */
ashrt_status ashrt_batch_forward(ashrt_batch* batch, const float* m_dev, float* d_dev, void* stream);
ashrt_status ashrt_batch_adjoint(ashrt_batch* batch, const float* d_dev, float* m_dev, void* stream);
/* robust_irls_deblend of every gather (opts masks must be NULL; reports has
 * ngather entries, may be NULL).  Requires with_solver.  Synchronises stream. */
ashrt_status ashrt_batch_deblend(ashrt_batch* batch, const float* d_dev, float* m_dev,
                                 float* drec_dev, const irls_opts* opts, irls_report* reports,
                                 void* stream);

/*
 * Measurement hooks (no counterpart in the paper; used to time the library's
 * own kernels on the streams they run on).
 *   ashrt_profile_enable(1): from now on every operator kernel launch is
 *     bracketed by two CUDA events recorded on its stream (cheap, but not free).
 *   ashrt_profile_read: synchronises on the recorded events and returns, per
 *     kernel class, the summed elapsed milliseconds and the number of timed
 *     launches since the previous read, then resets them.  Classes:
 *     0 model-side trace-axis r2c FFT (the forward's), 1 forward row kernel
 *     (t-FFT + Stolt map + sum), 2 adjoint row kernel, 3 model-side
 *     trace-axis c2r FFT (the adjoint's), 4 solver vector kernels (counted
 *     only), 5 data-side trace-axis r2c (the adjoint's), 6 data-side
 *     trace-axis c2r (the forward's).  n is the length of ms / launches (up
 *     to 7).
 *     Returns 0, or 1 if an event could not be read.
 *   ashrt_kernel_launches: total kernels this library has launched in the
 *     process (all classes, profiling on or off).
 */
void ashrt_profile_enable(int on);
int ashrt_profile_read(double* ms, long long* launches, int n);
long long ashrt_kernel_launches(void);

/*
 * FP32 CUDA-core peak of the current device, measured: the roofline
 * denominator of the ALU-bound row kernels (no counterpart in the paper).
 * Launches a kernel of independent FMA chains (8 per thread, 2048 threads per
 * SM on every SM) `reps` + 1 times on `stream` with `iters` loop trips each
 * (16 x 8 FMAs per trip and thread), times each launch with CUDA events and
 * returns the best rate after the first in *tflops (2 flops per FMA).
 * *sm_count (may be NULL) receives the device's SM count.  Synchronises the
 * stream; allocates no device memory.
 */
ashrt_status ashrt_fp32_peak(int iters, int reps, double* tflops, int* sm_count, void* stream);

/*
 * Deblending quality (ch. 4, Eqs ch4_Qpd and ch4_Qr), per gather:
 *   Q = 10 log10( ||d_orig||^2 / ||d_orig - d_test||^2 )  [dB]
 * with d_orig the unblended gather and d_test the pseudo-deblended one (Q_PD)
 * or the deblended one (Q_R); the improvement of a solve is Q_R - Q_PD.
 *   d_orig_dev, d_test_dev  [batch][n_per_gather] float32 (read)
 *   sums_dev   device array [batch][2] of double (written): sum d_orig^2 and
 *              sum (d_orig - d_test)^2, both accumulated in FP64
 *   q_db       host array [batch] (written; +inf where the gathers are equal,
 *              NaN where d_orig is all zero), or NULL: the call is then
 *              asynchronous on `stream` and leaves only sums_dev.  With q_db
 *              it synchronises `stream`.
 * batch <= 65535.  One kernel launch; no allocation.
 */
ashrt_status ashrt_quality_db(const float* d_orig_dev, const float* d_test_dev, int batch,
                              long long n_per_gather, double* sums_dev, double* q_db,
                              void* stream);

/*
 * Learned warm start (no counterpart in the paper, which starts every solve
 * from m = 0 and W = I): a 4-level convolutional U-Net that maps a
 * pseudo-deblended gather (an H x W = nx x nt image) to out_channels maps on
 * the same grid -- the P model panels of the initial Radon model and the log
 * of the initial residual weights -- trained on pairs the robust solve itself
 * produces.  Channels per level 16, 48, 96, 192; 3x3 convolutions with ReLU,
 * 2x2 average pooling, nearest 2x upsampling, skip concatenation, 1x1 head.
 * BF16 weights and activations, FP32 accumulation, FP32 master weights and
 * gradients, Adam (beta 0.9, 0.999, eps 1e-8).
 *   ashrt_unet_create: H, W multiples of 8; max_batch images per call; the
 *     parameters are init_params (n_init values, layer by layer: weights
 *     [cout][cin][k][k] then biases [cout]) or, if NULL, He-normal from a fixed
 *     seed.  Allocates all device memory here (ENOMEM on failure).
 *   ashrt_unet_param_count: number of parameters.
 *   ashrt_unet_get: copies parameters and/or gradients of the last training
 *     step to host arrays (either may be NULL); synchronises the device.
 *   ashrt_unet_forward: x_dev [n][H][W] fp32 -> y_dev [n][out_channels][H][W]
 *     fp32.  Each input is divided by its RMS; with rescale = 0 the outputs
 *     stay in these normalised units, with rescale = 1 they are returned in
 *     input units for an IRLS misfit power p (panels times the RMS, the last
 *     channel as exp(y) RMS^((p-2)/2)).  Async on stream.
 *   ashrt_unet_train_step: one Adam step (lr > 0; lr = 0 only computes the
 *     gradients) on n pairs, targets t_dev [n][out_channels][H][W] in
 *     normalised units, loss sum_c w_c mean (y_c - t_c)^2 with host weights
 *     channel_weight[out_channels] (NULL = 1); *loss (may be NULL) receives
 *     the loss before the step, which synchronises the stream.
 * The convolutions run on the tensor cores (tcgen05 for the forward pass and
 * the input gradients, mma.sync for the weight gradients); their device-side
 * waits are bounded, and one that ran out is reported as ASHRT_ETIMEOUT by the
 * next synchronising call (ashrt_unet_train_step with a loss, ashrt_unet_get).
 * Device pointers are caller-owned; all return EINVAL on bad sizes.
 */
typedef struct ashrt_unet ashrt_unet;
ashrt_status ashrt_unet_create(ashrt_unet** out, int H, int W, int out_channels, int max_batch,
                               const float* init_params, long long n_init);
void ashrt_unet_destroy(ashrt_unet* net);
long long ashrt_unet_param_count(const ashrt_unet* net);
ashrt_status ashrt_unet_get(const ashrt_unet* net, float* params, float* grads, long long n);
ashrt_status ashrt_unet_forward(ashrt_unet* net, const float* x_dev, float* y_dev, int n,
                                int rescale, float p, void* stream);
ashrt_status ashrt_unet_train_step(ashrt_unet* net, const float* x_dev, const float* t_dev, int n,
                                   const float* channel_weight, float lr, double* loss,
                                   void* stream);
/* Training targets in the network's units from a solve (robust_irls_deblend
 * with wr_out_dev) of the gathers x_dev [n][H][W]: its model m_dev
 * [n][out_channels-1][H][W] divided by the RMS of x, and log wr_dev [n][H][W]
 * minus (p-2)/2 log RMS, into t_dev [n][out_channels][H][W].  Async. */
ashrt_status ashrt_unet_targets(ashrt_unet* net, const float* x_dev, const float* m_dev,
                                const float* wr_dev, float* t_dev, int n, float p, void* stream);
/* The warm start of robust_irls_deblend for gathers x_dev [n][H][W]: the
 * network's prediction in input units, model m0_dev [n][out_channels-1][H][W]
 * and residual weights wr0_dev [n][H][W] (either may be NULL).  Async. */
ashrt_status ashrt_unet_predict(ashrt_unet* net, const float* x_dev, float* m0_dev,
                                float* wr0_dev, int n, float p, void* stream);

/* Text of the last error raised on the calling thread ("" if none). */
const char* ashrt_last_error(void);

/* Static name of a status code. */
const char* ashrt_status_string(ashrt_status s);

#ifdef __cplusplus
}
#endif

#endif /* ASHRT_H */
