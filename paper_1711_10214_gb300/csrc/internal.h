// Host-side declarations shared by the translation units of libashrt.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "ashrt.h"

namespace ashrt {

// Arguments of the x-direction (trace-axis) transforms.  One "slab" is one
// [nx][nt] real panel and its [Lh][ld] complex half spectrum in k_x.
struct XfftArgs {
  const float* in_real = nullptr;    // r2c input  [slabs][nx][nt]
  float2* out_cplx = nullptr;        // r2c output [slabs][Lh][ld]
  const float2* in_cplx = nullptr;   // c2r input  [slabs][Lh][ld]
  float* out_real = nullptr;         // c2r output [slabs][nx][nt]
  int nx = 0, nt = 0, ld = 0, Lh = 0, Nx = 0;
  long long slab_real = 0;           // nx * nt
  long long slab_cplx = 0;           // Lh * ld
  const float* ew = nullptr;         // elementwise weight on the real side, or null
  const float* tmask = nullptr;      // per-trace weight [gather][nx], or null
  int slabs_per_gather = 1;
  double* dot = nullptr;             // c2r: per-gather sum of squared outputs (added), or null
  int ew_sq = 0;                     // c2r: store out * ew^2 (dot still sums (out * ew)^2)
  const float2* tw = nullptr;        // base twiddles of length Nx
  int slabs = 0;
  int cols = 16;                     // complex time columns per CTA: 16 or 8 (Nx <= 512)
  // r2c only: a CGLS vector update fused into the input load (the solver's
  // mu = 0 path).  Per gather g, coef[g] = (cs, beta, alpha, alpha2):
  //   mode 1 (model side): x = cs s + beta p; p_out <- x;
  //                        u <- u + alpha p (+ alpha2 p2 when cg_p2_read)
  //   mode 2 (data side):  x = r - alpha q;  r <- x
  // where p (mode 1) or r (mode 2) is in_real, and x is then transformed.
  // p_out is cg_pout, or in_real itself (in place) when cg_pout is null; p2
  // (read only when cg_p2_read) is the same buffer as cg_pout: a p two
  // iterations old whose elements are read before x overwrites them.
  int cg_mode = 0;
  float* cg_io = nullptr;            // == in_real
  const float* cg_s = nullptr;       // s (mode 1) or q (mode 2)
  float* cg_u = nullptr;             // u (mode 1)
  float* cg_pout = nullptr;          // mode 1: where x is written (null: in place)
  int cg_p2_read = 0;                // mode 1: add alpha2 p2, p2 read from cg_pout
  int cg_u_rw = 1;                   // mode 1: u is updated (0: u is neither read nor written)
  const float4* cg_coef = nullptr;   // [gathers]
  int tma = 1;                       // r2c: use the persistent TMA kernel where it applies
  int* err = nullptr;                // set to 1 if a bounded device wait ran out
};

// A CGLS update to fuse into an operator's first (r2c) transform.
struct CgFuse {
  int mode = 0;                      // 1: model side (forward), 2: data side (adjoint)
  int model_ew_sq = 0;               // adjoint: the model-side output is stored times ew_model
                                     // once more (W_m^-2 L^T ..., the CG's s~ = W_m^-1 s)
  const float* s = nullptr;          // s (mode 1) or q (mode 2)
  float* u = nullptr;                // u (mode 1)
  float* pout = nullptr;             // mode 1: the new p's buffer (null: in place)
  int p2_read = 0;                   // mode 1: also add alpha2 times the p held in pout
  int u_rw = 1;                      // mode 1: this launch updates u (0: u untouched)
  const float4* coef = nullptr;      // per gather (cs, beta, alpha, alpha2)
};

// Arguments of the fused t-FFT + Stolt map + sum/spray row kernels.
struct RowArgs {
  const float2* X = nullptr;   // model spectra [B][P][Lh][ld]  (fwd in / adj out)
  float2* Xw = nullptr;
  const float2* Y = nullptr;   // data spectrum [B][Lh][ld]     (adj in / fwd out)
  float2* Yw = nullptr;
  int nt = 0, ld = 0, Lh = 0, P = 0, nv = 0, nt0 = 0, Nt = 0;
  long long x_batch = 0, x_panel = 0, y_batch = 0;
  const float2* tw = nullptr;      // base twiddles of length Nt
  const float2* tw16 = nullptr;    // the same for the radix-16 schedule (stolt_r16.cu), or null
  const float* wt = nullptr;       // [Nt] spectral weight W(w)/(Nt Nx), 0 at unmapped bins
  const int* kmin = nullptr;       // [nv][Lh] first mapped |k| (host FP64 cone rule)
  const float2* acone = nullptr;   // [nv][Lh] cone parameter a as (hi, lo) floats
  const unsigned* taps = nullptr;  // [nv][Lh][taps_ld] Stolt taps of |k| (see tap_word)
  int taps_ld = 0;                 // words per (v, l) row: Nt/2 + 1 rounded up to 4
  const uint2* atab = nullptr;     // [nv][Lh][atab_ld] adjoint source table (see build_adj_table)
  int atab_ld = 0;                 // entries per (v, l) row: Nt/2 + 1 rounded up to 2
  const float2* phase = nullptr;   // [nt0][Nt] exp(-i w tau0), or null (tau0 == 0)
  int batch = 0;
  int minb = 3;                    // variant: 1, 2, 3 radix-8 kernels capped for that many
                                   // resident CTAs per SM; 4 radix-16 forward, radix-8
                                   // adjoint; 5 radix-16 both; 6 single-gather radix-16
                                   // both; 7 single-gather radix-16 forward, radix-8
                                   // adjoint; 8 radix-16 pair forward, single-gather
                                   // radix-16 adjoint; 9 as 5 with the forward's
                                   // accumulator in tensor memory (4..9 need tw16)
};

cudaError_t launch_xfft_r2c(const XfftArgs& a, cudaStream_t s);
cudaError_t launch_xfft_c2r(const XfftArgs& a, cudaStream_t s);
cudaError_t launch_stolt_fwd_rows(const RowArgs& a, cudaStream_t s);
cudaError_t launch_stolt_adj_rows(const RowArgs& a, cudaStream_t s);
// Radix-16 row kernels (Nt = 1024, 2048, 4096 only; see stolt_r16.cu).
bool rows16_supported(int logNt);
cudaError_t launch_stolt_fwd_rows16(const RowArgs& a, cudaStream_t s);
cudaError_t launch_stolt_fwd_rows16_tm(const RowArgs& a, cudaStream_t s);
cudaError_t launch_stolt_adj_rows16(const RowArgs& a, cudaStream_t s);
// Single-gather radix-16 row kernels (Nt = 1024, 2048, 4096; see stolt_r16s.cu).
cudaError_t launch_stolt_fwd_rows16s(const RowArgs& a, cudaStream_t s);
cudaError_t launch_stolt_adj_rows16s(const RowArgs& a, cudaStream_t s);

// Stolt tap table: one 32-bit word per (velocity, k_x index l, |k|), |k| in
// [0, Nt/2].  Mapped bins hold (floor(u) << 20) | round(frac(u) 2^20) with
// u = sqrt(k^2 - a^2) evaluated in FP64 (a as in the cone rule); unmapped bins
// (k^2 <= a^2, or |k| = Nt/2) hold kTapInvalid.
constexpr unsigned kTapInvalid = 0xffffffffu;
inline int taps_row_len(int Nt) { return ((Nt / 2 + 1) + 3) & ~3; }
void build_tap_rows(const float* velocities, int nv, int Nt, int Nx, int Lh, double dt, double dx,
                    unsigned* taps, int* kmin, float2* acone);
// Source table of the transposed map (the adjoint's gather), one row per
// (velocity, l), entries J in [0, Nt/2].  With ks[J] the first |k| >= kmin
// whose tap floor index (word >> 20) is >= J, bin J of the w_tau spectrum
// takes (1 - f(kB)) D(kB) from its primary source kB = ks[J] when
// floor(u(kB)) = J, and f(kB - 1) D(kB - 1) from its secondary source
// kB - 1 when floor(u(kB - 1)) = J - 1, f being the tap fraction.  Since
// u(k + 1) - u(k) = (2k + 1) / (u(k + 1) + u(k)) >= 1, floor(u) is strictly
// increasing in k: a bin has at most one source of each kind.  Entry
// x = frac20(kB) | kB << 20, y = frac20(kB - 1) | has_primary << 20 |
// has_secondary << 21 (both fractions and indices taken from the tap words,
// so both directions of the map use the same taps).  Rows with
// kmin >= Nt/2 are zero.  Returns false if a bin had two sources of one kind.
inline int atab_row_len(int Nt) { return ((Nt / 2 + 1) + 1) & ~1; }
bool build_adj_table(const unsigned* taps, const int* kmin, int nv, int Lh, int Nt, uint2* atab);

// Traces at irregular positions (irregular.cu): the data-side trace-axis
// synthesis d = Re(Es Y) and analysis Yhat = Ea d as dense contractions.
// Es [nr][Lh] = c_l exp(+2 pi i l x_j / (Nx dx)) (c_l = 2 but 1 at l = 0 and
// Nx/2; the Nyquist row is cos(pi x_j / dx)); Ea [Lh][nr] = conj of the same
// without c_l.  Returns false on a non-finite position.
bool build_irregular_tables(const double* x, int nr, int Nx, double dx, float2* Es, float2* Ea);
cudaError_t launch_irr_synth(const float2* Es, const float2* Y, float* d, int nr, int nt, int Lh,
                             int ld, long long y_batch, const float* ew, const float* tmask,
                             double* dot, int batch, cudaStream_t s);
cudaError_t launch_irr_analysis(const float2* Ea, const float* d, float2* Yh, int nr, int nt,
                                int Lh, int ld, long long y_batch, const float* ew,
                                const float* tmask, int batch, cudaStream_t s);
cudaError_t launch_irr_cg_r(float* r, const float* q, long long n, const float4* coef, int batch,
                            cudaStream_t s);

// Twiddle tables in the layout the device passes expect (see common.cuh):
// radix 2^lr passes while lr or more factors of two remain, then one smaller
// radix (lr = 3 for the radix-8 kernels, 4 for the radix-16 row kernels).
int twiddle_table_len(int logn, int lr = 3);
void build_twiddle_table(int logn, float2* out, int lr = 3);

void set_error(const char* fmt, ...);

// Launch accounting / optional event timing per kernel class (prof.cu).
// PROF_XR2C / PROF_XC2R: the model-side trace-axis transforms (forward r2c,
// adjoint c2r); the data-side ones (one row per gather) have their own classes.
enum ProfClass { PROF_XR2C = 0, PROF_ROWS_FWD = 1, PROF_ROWS_ADJ = 2, PROF_XC2R = 3,
                 PROF_SOLVER = 4, PROF_XR2C_DATA = 5, PROF_XC2R_DATA = 6, kProfClasses = 7 };
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s);
void count_launches(int n);
// While a stream capture is being recorded on this thread, launches are
// counted into the capture (returned by prof_capture_end) and not timed.
void prof_capture_begin();
long long prof_capture_end();

// Arguments a recorded solve graph was captured with.
struct GraphKey {
  const float* d = nullptr;
  const float* m = nullptr;
  const float* drec = nullptr;
  int B = 0;
  irls_opts opts{};
  bool operator==(const GraphKey& o) const {
    const irls_opts &a = opts, &b = o.opts;
    return d == o.d && m == o.m && drec == o.drec && B == o.B && a.p == b.p && a.q == b.q &&
           a.n_outer == b.n_outer && a.n_cg == b.n_cg && a.tol == b.tol && a.b_r == b.b_r &&
           a.b_m == b.b_m && a.mu == b.mu && a.warm_start_cg == b.warm_start_cg &&
           a.eps_r_fixed == b.eps_r_fixed && a.eps_m_fixed == b.eps_m_fixed &&
           a.trace_mask_dev == b.trace_mask_dev && a.apex_mask_dev == b.apex_mask_dev &&
           a.m0_dev == b.m0_dev && a.wr0_dev == b.wr0_dev && a.wr_out_dev == b.wr_out_dev;
  }
};

}  // namespace ashrt

// The plan (opaque to users).
struct ashrt_plan {
  int device = 0;
  int nt = 0, nx = 0, nv = 0, nt0 = 0, P = 0;
  int nr = 0;                // data traces per gather (= nx unless the traces are irregular)
  bool irregular = false;    // data traces at given positions (Es / Ea below)
  double dt = 0, dx = 0;
  int Nt = 0, Nx = 0, Lh = 0, ld = 0, logNt = 0, logNx = 0;
  int max_batch = 1;
  int with_solver = 0;
  ashrt_opts opts{};
  bool shift = false;        // any nonzero tau0
  int rows_minb = 3;         // row-kernel variant 1..9 (autotuned; see ashrt_plan_autotune)
  int xfft_cols = 16;
  // device tables
  float2* tw_t = nullptr;
  float2* tw_t16 = nullptr;  // radix-16 schedule of length Nt (rows16_supported), else null
  float2* tw_x = nullptr;
  float* wt = nullptr;
  int* kmin = nullptr;
  float2* acone = nullptr;
  unsigned* taps = nullptr;
  uint2* atab = nullptr;
  float2* phase = nullptr;
  float2* Es = nullptr;      // irregular traces: synthesis table [nr][Lh]
  float2* Ea = nullptr;      // irregular traces: analysis table [Lh][nr]
  // workspace
  float2* X = nullptr;       // [max_batch][P][Lh][ld]
  float2* Y = nullptr;       // [max_batch][Lh][ld]
  size_t ws_bytes = 0;
  // solver vectors (with_solver)
  float* u = nullptr;        // model-sized
  float* pv = nullptr;       // model-sized
  float* sv = nullptr;       // model-sized
  float* wminv = nullptr;    // model-sized
  float* r = nullptr;        // data-sized
  float* qv = nullptr;       // data-sized
  float* wr = nullptr;       // data-sized
  float* y = nullptr;        // data-sized
  float4* cg_coef = nullptr; // [2][max_batch] fused CGLS coefficients (forward, adjoint)
  int* dev_err = nullptr;    // set by a device wait that ran out (checked by the solver)
  double* scal = nullptr;    // per-gather scalars
  unsigned int* sel = nullptr;   // per-gather selection scratch
  int* flags = nullptr;      // per-gather status flags
  // recorded solve (robust_irls_deblend with use_graph)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  ashrt::GraphKey graph_key;
  long long graph_kernels = 0;
  int graph_applies_f = 0, graph_applies_a = 0;
};
