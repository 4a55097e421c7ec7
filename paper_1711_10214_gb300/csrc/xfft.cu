// Trace-axis (x) transforms of the Stolt ASHRT: the F_x part of the 2-D
// Fourier transforms F of ch. 5 Eqs ch5_forward_operator / ch5_adj_operator.
//
//   r2c: a real [nx][nt] panel, zero-padded to Nx traces, -> its half spectrum
//        in k_x, [Lh = Nx/2 + 1][nt] complex (analysis, exp(-i k_x x)).
//   c2r: a Hermitian half spectrum [Lh][nt] -> the real panel, synthesis
//        exp(+i k_x x), unnormalised, cropped to nx traces.
//
// One CTA transforms 2*C consecutive time columns of one panel: adjacent
// columns t, t+1 are packed as the real and imaginary parts of one complex
// sequence (one 8-byte load per trace), transformed together, and separated
// with the Hermitian symmetry of real signals (one 16-byte store per row).  The length-Nx transforms run as Stockham passes
// over a shared [Nx][C] tile; the first pass is fed straight from global
// memory and (c2r) the last pass stores straight to global memory.  The
// per-element weights of the IRLS operator (W_m^-1 on the model side,
// W_r and the sampling mask on the data side) are fused into those loads and
// stores, and the c2r kernel can also accumulate the FP64 sum of squares of
// what it stores (the CGLS norms) per gather.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace ashrt {

namespace {

template <int DIR, int N, int C, int R>
__device__ __forceinline__ void col_pass(float2* sm, int Ns, const float2* __restrict__ tw,
                                         int off, int tid) {
  constexpr int T = N * C / 16, NB = 16 / R, JS = T / C;
  const int col = tid % C, j0 = tid / C;
  float2 v[16];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = j0 + JS * q;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = sm[(jb + r * (N / R)) * C + col];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = j0 + JS * q;
    const int k = jb & (Ns - 1);
    if (Ns > 1) twiddle_r<R>(&v[q * R], base_twiddle<DIR>(tw, off, k));
    dft_r<DIR, R>(&v[q * R]);
    const int base = (jb - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) sm[(base + r * Ns) * C + col] = v[q * R + r];
  }
  __syncthreads();
}

template <int DIR, int LOGN, int C, int Q0, int Q1>
__device__ __forceinline__ void col_pass_range(float2* sm, const float2* __restrict__ tw, int tid) {
  using S = Sched<LOGN>;
  if constexpr (Q0 < Q1) {
    col_pass<DIR, S::N, C, S::radix(Q0)>(sm, S::ns(Q0), tw, S::tw_off(Q0), tid);
    col_pass_range<DIR, LOGN, C, Q0 + 1, Q1>(sm, tw, tid);
  }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Adds the CTA-wide sum of `part` to *dst (one atomic per CTA).
__device__ __forceinline__ void block_accumulate(double part, double* dst) {
  __shared__ double red[32];
  part = warp_sum(part);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double x = lane < nw ? red[lane] : 0.0;
    x = warp_sum(x);
    if (lane == 0) atomicAdd(dst, x);
  }
}

// Real time samples t and t+1 of one trace, packed as z = x_t + i x_{t+1}
// (one 8-byte load when the row is 8-byte aligned).
__device__ __forceinline__ float2 load_pair_real(const float* __restrict__ row, int t, int nt,
                                                 bool vec) {
  if (vec && t + 1 < nt) return __ldg((const float2*)(row + t));
  return make_float2(t < nt ? __ldg(row + t) : 0.f, t + 1 < nt ? __ldg(row + t + 1) : 0.f);
}

// Plain (coherent) pair load / store of samples t, t+1 of a row, for the
// in-place CGLS updates (each pair is read and written by one thread).
__device__ __forceinline__ float2 ld_pair(const float* row, int t, int nt, bool vec) {
  if (vec && t + 1 < nt) return *(const float2*)(row + t);
  return make_float2(t < nt ? row[t] : 0.f, t + 1 < nt ? row[t + 1] : 0.f);
}

__device__ __forceinline__ void st_pair(float* row, int t, int nt, bool vec, float2 v) {
  if (vec && t + 1 < nt) {
    *(float2*)(row + t) = v;
    return;
  }
  if (t < nt) row[t] = v.x;
  if (t + 1 < nt) row[t + 1] = v.y;
}

// The fused CGLS update of one sample pair (see XfftArgs::cg_mode); returns
// the updated vector's pair, which is what the transform consumes.
__device__ __forceinline__ float2 cg_update_pair(const XfftArgs& a, long long off, int t, bool vec,
                                                 float4 cf) {
  float* io = a.cg_io + off;
  const float2 x = ld_pair(io, t, a.nt, vec);
  const float2 y = ld_pair(a.cg_s + off, t, a.nt, vec);
  float2 z;
  if (a.cg_mode == 1) {
    float* po = a.cg_pout ? a.cg_pout + off : io;
    z = make_float2(fmaf(cf.x, y.x, cf.y * x.x), fmaf(cf.x, y.y, cf.y * x.y));
    const bool two = a.cg_p2_read && cf.w != 0.f;
    if (a.cg_u_rw && (cf.z != 0.f || two)) {
      float* u = a.cg_u + off;
      float2 un = ld_pair(u, t, a.nt, vec);
      if (two) {
        const float2 p2 = ld_pair(po, t, a.nt, vec);   // read before z overwrites it
        un = make_float2(fmaf(cf.w, p2.x, un.x), fmaf(cf.w, p2.y, un.y));
      }
      un = make_float2(fmaf(cf.z, x.x, un.x), fmaf(cf.z, x.y, un.y));
      st_pair(u, t, a.nt, vec, un);
    }
    st_pair(po, t, a.nt, vec, z);
  } else {
    z = make_float2(fmaf(-cf.z, y.x, x.x), fmaf(-cf.z, y.y, x.y));
    st_pair(io, t, a.nt, vec, z);
  }
  return z;
}

template <int LOGN, int C>
__global__ void __launch_bounds__((1 << LOGN) * C / 16)
xfft_r2c_kernel(XfftArgs a) {
  constexpr int N = 1 << LOGN, T = N * C / 16, JS = T / C;
  using S = Sched<LOGN>;
  extern __shared__ float2 sm[];   // [N][C]
  const int tid = threadIdx.x, col = tid % C, j0 = tid / C;
  const long long slab = blockIdx.x;
  const int t0 = blockIdx.y * 2 * C;
  const int ta = t0 + 2 * col;      // this thread packs columns ta (real) and ta + 1 (imag)
  const bool vec = (a.nt & 1) == 0;
  const float* in = a.in_real + slab * a.slab_real;
  const float* ew = a.ew ? a.ew + slab * a.slab_real : nullptr;
  const float* tm = a.tmask ? a.tmask + (slab / a.slabs_per_gather) * a.nx : nullptr;
  const float4 cf = a.cg_mode ? a.cg_coef[slab / a.slabs_per_gather] : make_float4(0.f, 0.f, 0.f, 0.f);

  // first pass (radix 8, Ns = 1) for both butterflies of this thread: all
  // loads first; rows >= nx are the zero padding
  float2 v[2][8];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int jb = j0 + JS * q;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = jb + r * (N / 8);
      float2 z = make_float2(0.f, 0.f);
      if (row < a.nx) {
        const long long o = (long long)row * a.nt;
        z = a.cg_mode ? cg_update_pair(a, slab * a.slab_real + o, ta, vec, cf)
                      : load_pair_real(in + o, ta, a.nt, vec);
        if (ew) {
          const float2 w = load_pair_real(ew + o, ta, a.nt, vec);
          z.x *= w.x;
          z.y *= w.y;
        }
        if (tm) {
          const float g = __ldg(tm + row);
          z.x *= g;
          z.y *= g;
        }
      }
      v[q][r] = z;
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int jb = j0 + JS * q;
    dft8<-1>(v[q]);
#pragma unroll
    for (int r = 0; r < 8; ++r) sm[(jb * 8 + r) * C + col] = v[q][r];
  }
  __syncthreads();
  col_pass_range<-1, LOGN, C, 1, S::NPASS>(sm, a.tw, tid);

  // separate the packed columns: A = (Z_l + conj Z_{N-l}) / 2 (column ta),
  // B = (Z_l - conj Z_{N-l}) / (2i) (column ta + 1), 0 <= l <= N/2; one
  // 16-byte store of (A, B) per row
  float2* out = a.out_cplx + slab * a.slab_cplx;
  for (int f = tid; f < (N / 2 + 1) * C; f += T) {
    const int l = f / C, c = f % C;
    const float2 zl = sm[l * C + c];
    const float2 zm = sm[((N - l) & (N - 1)) * C + c];
    const float4 AB = make_float4(0.5f * (zl.x + zm.x), 0.5f * (zl.y - zm.y),
                                  0.5f * (zl.y + zm.y), -0.5f * (zl.x - zm.x));
    const int t = t0 + 2 * c;
    float2* o = out + (long long)l * a.ld + t;
    if (t + 1 < a.nt) {
      *(float4*)o = AB;
    } else if (t < a.nt) {
      o[0] = make_float2(AB.x, AB.y);
    }
  }
}

// Persistent TMA variant of the r2c transform: 16 real time columns (C = 8
// packed pairs) per tile, one CTA loops over tiles.  The input tile of every
// vector the load needs (the transformed vector, and for the fused CGLS
// update s / q and u, and the weight) is brought into shared memory by TMA
// box loads [nx][16] that signal one mbarrier; as soon as the first pass has
// consumed the staged tile (and the fused update has been written back by
// TMA stores), the next tile's loads are issued, so they overlap the
// remaining FFT passes and the spectrum stores of the current tile.
// Requires nx <= 256 (one box per vector), nt % 4 == 0 and 16-byte aligned
// vectors; the launcher falls back to xfft_r2c_kernel otherwise.
struct R2cMaps {
  CUtensorMap in, s, u, w, p2;   // p2: the new p's buffer (cg_pout), also read when cg_p2_read
};

template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 2)
xfft_r2c_tma(XfftArgs a, const __grid_constant__ R2cMaps mp, int n_tt, long long n_tiles) {
  constexpr int N = 1 << LOGN, C = 8, T = N * C / 16, JS = T / C;
  using S = Sched<LOGN>;
  extern __shared__ unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 127) & ~(uintptr_t)127);
  const int mode = a.cg_mode;
  const bool has_w = a.ew != nullptr;
  const int box = a.nx * 16;                          // floats of one vector's box
  const int slot = (box * 4 + 127) & ~127;            // bytes, 128-byte aligned
  const bool p2r = mode == 1 && a.cg_p2_read;
  const bool urw = mode == 1 && a.cg_u_rw;
  const bool pout = mode == 1 && a.cg_pout != nullptr;
  const int i_s = 1, i_u = 2, i_p2 = urw ? 3 : 2;
  const int i_w = 1 + (mode ? 1 : 0) + (urw ? 1 : 0) + (p2r ? 1 : 0);
  const int nslot = i_w + (has_w ? 1 : 0);
  float* st_in = (float*)base;
  float* st_s = (float*)(base + i_s * slot);
  float* st_u = (float*)(base + i_u * slot);
  float* st_p2 = (float*)(base + i_p2 * slot);
  float* st_w = (float*)(base + i_w * slot);
  float2* sm = (float2*)(base + nslot * slot);        // [N][C]
  uint64_t* bar = (uint64_t*)(sm + N * C);
  const int tid = threadIdx.x, col = tid % C, j0 = tid / C;

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](long long tile) {
    const int z = (int)(tile / n_tt), x = (int)(tile % n_tt) * 16;
    mbar_arrive_expect_tx(bar, (uint32_t)(nslot * box * 4));
    tma_load_3d(st_in, &mp.in, x, 0, z, bar);
    if (mode) tma_load_3d(st_s, &mp.s, x, 0, z, bar);
    if (urw) tma_load_3d(st_u, &mp.u, x, 0, z, bar);
    if (p2r) tma_load_3d(st_p2, &mp.p2, x, 0, z, bar);
    if (has_w) tma_load_3d(st_w, &mp.w, x, 0, z, bar);
  };
  long long tile = blockIdx.x;
  if (tile < n_tiles && tid == 0) issue(tile);
  uint32_t parity = 0;
  for (; tile < n_tiles; tile += gridDim.x) {
    const long long slab = tile / n_tt;
    const int t0 = (int)(tile % n_tt) * 16;
    const long long g = slab / a.slabs_per_gather;
    const float* tm = a.tmask ? a.tmask + g * a.nx : nullptr;
    const float4 cf = mode ? a.cg_coef[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool ok = mbar_wait_bounded(bar, parity);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        if (a.err) atomicExch(a.err, 1);
        bulk_wait_all();
      }
      return;
    }
    parity ^= 1u;

    // first pass from the staged tile (fused update written back in place)
    float2 v[2][8];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int jb = j0 + JS * q;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int row = jb + r * (N / 8);
        float2 z = make_float2(0.f, 0.f);
        if (row < a.nx) {
          const int e = row * 16 + 2 * col;
          float2 x = *(const float2*)(st_in + e);
          if (mode == 1) {
            const float2 sv = *(const float2*)(st_s + e);
            const bool two = p2r && cf.w != 0.f;
            if (urw && (cf.z != 0.f || two)) {
              float2 un = *(const float2*)(st_u + e);
              if (two) {
                const float2 p2 = *(const float2*)(st_p2 + e);
                un = make_float2(fmaf(cf.w, p2.x, un.x), fmaf(cf.w, p2.y, un.y));
              }
              *(float2*)(st_u + e) = make_float2(fmaf(cf.z, x.x, un.x), fmaf(cf.z, x.y, un.y));
            }
            x = make_float2(fmaf(cf.x, sv.x, cf.y * x.x), fmaf(cf.x, sv.y, cf.y * x.y));
            *(float2*)(st_in + e) = x;
          } else if (mode == 2) {
            const float2 qv = *(const float2*)(st_s + e);
            x = make_float2(fmaf(-cf.z, qv.x, x.x), fmaf(-cf.z, qv.y, x.y));
            *(float2*)(st_in + e) = x;
          }
          if (has_w) {
            const float2 w = *(const float2*)(st_w + e);
            x.x *= w.x;
            x.y *= w.y;
          }
          if (tm) {
            const float gm = __ldg(tm + row);
            x.x *= gm;
            x.y *= gm;
          }
          z = x;
        }
        v[q][r] = z;
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int jb = j0 + JS * q;
      dft8<-1>(v[q]);
#pragma unroll
      for (int r = 0; r < 8; ++r) sm[(jb * 8 + r) * C + col] = v[q][r];
    }
    if (mode) fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      if (mode) {
        tma_store_3d(pout ? &mp.p2 : &mp.in, t0, 0, (int)slab, st_in);
        if (urw && (cf.z != 0.f || (p2r && cf.w != 0.f)))
          tma_store_3d(&mp.u, t0, 0, (int)slab, st_u);
        bulk_commit();
        bulk_wait_read();
      }
      const long long nxt = tile + gridDim.x;
      if (nxt < n_tiles) {
        fence_proxy_async();
        issue(nxt);
      }
    }
    col_pass_range<-1, LOGN, C, 1, S::NPASS>(sm, a.tw, tid);

    float2* out = a.out_cplx + slab * a.slab_cplx;
    for (int f = tid; f < (N / 2 + 1) * C; f += T) {
      const int l = f / C, c = f % C;
      const float2 zl = sm[l * C + c];
      const float2 zm = sm[((N - l) & (N - 1)) * C + c];
      const float4 AB = make_float4(0.5f * (zl.x + zm.x), 0.5f * (zl.y - zm.y),
                                    0.5f * (zl.y + zm.y), -0.5f * (zl.x - zm.x));
      const int t = t0 + 2 * c;
      float2* o = out + (long long)l * a.ld + t;
      if (t + 1 < a.nt) {
        *(float4*)o = AB;
      } else if (t < a.nt) {
        o[0] = make_float2(AB.x, AB.y);
      }
    }
    __syncthreads();
  }
  if (tid == 0) bulk_wait_all();
}

// Stored row `row` (<= N/2) of the half spectrum for the two adjacent columns
// t and t+1 (t even): (A, B) = (re, im of column t, re, im of column t+1).
// Rows are ld >= nt long with ld a multiple of 4, so the 16-byte load at an
// even t < nt stays inside the row; a column >= nt reads as zero.
__device__ __forceinline__ float4 col_load2(const float2* __restrict__ base, int ld, int row, int t,
                                            int nt) {
  const bool ok = t < nt, okb = t + 1 < nt;
  const float4 y = __ldg((const float4*)(base + (long long)row * ld + (ok ? t : 0)));
  return make_float4(ok ? y.x : 0.f, ok ? y.y : 0.f, okb ? y.z : 0.f, okb ? y.w : 0.f);
}
// Z = A + i B of a stored row (zdir), of its mirror N - row, whose A and B
// are the conjugates (zmir), and of rows 0 and N/2, whose imaginary parts a
// real signal's spectrum does not have (zreal).
__device__ __forceinline__ float2 zdir(float4 y) { return make_float2(y.x - y.w, y.y + y.z); }
__device__ __forceinline__ float2 zmir(float4 y) { return make_float2(y.x + y.w, y.z - y.y); }
__device__ __forceinline__ float2 zreal(float4 y) { return make_float2(y.x, y.z); }

// PF: the tile of the elementwise weight ew that this CTA's outputs use
// ([nx][2C] floats) is copied into shared memory with cp.async when the CTA
// starts, so the epilogue reads it from there instead of waiting on global
// loads after the transform (host condition: nt a multiple of 4, the tile
// fits; 16-byte chunks wholly inside the row are copied, the rest are never
// read).  NXH: nx <= N/2, so outputs r >= R/2 of every last-pass butterfly
// (traces jb + r N/R >= N/2) are cropped away and are not formed.
template <int LOGN, int C, bool PF, bool NXH>
__global__ void __launch_bounds__((1 << LOGN) * C / 16)
xfft_c2r_kernel(XfftArgs a) {
  constexpr int N = 1 << LOGN, T = N * C / 16, JS = T / C;
  using S = Sched<LOGN>;
  extern __shared__ float2 sm[];   // [N][C], then (PF) the weight tile [nx][2C] floats
  const int tid = threadIdx.x, col = tid % C, j0 = tid / C;
  const long long slab = blockIdx.x;
  const int t0 = blockIdx.y * 2 * C;
  const int ta = t0 + 2 * col;
  const float2* in = a.in_cplx + slab * a.slab_cplx;
  float* sew = (float*)(sm + N * C);
  if (PF) {
    const float* ews = a.ew + slab * a.slab_real;
    constexpr int CPR = C / 2;                   // 16-byte chunks per tile row
    for (int c = tid; c < a.nx * CPR; c += T) {
      const int row = c / CPR, q = c % CPR, t = t0 + 4 * q;
      if (t < a.nt) cp_async16(sew + row * 2 * C + 4 * q, ews + (long long)row * a.nt + t);
    }
    cp_async_commit();
  }

  // first pass (radix 8: butterfly jb takes rows jb + r N/8) on Z = A + i B,
  // A and B the Hermitian-extended spectra of columns ta, ta + 1.  Row
  // jb + r N/8 > N/2 mirrors row (N/8 - jb) + (7 - r) N/8, so the thread
  // takes butterflies jb and N/8 - jb together and builds their 16 inputs
  // from 8 stored rows (jb = 0 pairs with N/16 = JS, each its own mirror:
  // 9 rows, the Nyquist row included).
  float2 v[2][8];
  const int jb0 = j0, jb1 = j0 == 0 ? JS : N / 8 - j0;
  {
    float4 ya[4], yb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      ya[r] = col_load2(in, a.ld, jb0 + r * (N / 8), ta, a.nt);
      yb[r] = col_load2(in, a.ld, jb1 + r * (N / 8), ta, a.nt);
    }
    if (j0 == 0) {
      const float4 yn = col_load2(in, a.ld, N / 2, ta, a.nt);
      v[0][0] = zreal(ya[0]);
      v[0][4] = zreal(yn);
#pragma unroll
      for (int r = 1; r < 4; ++r) {
        v[0][r] = zdir(ya[r]);
        v[0][8 - r] = zmir(ya[r]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        v[0][r] = zdir(ya[r]);
        v[0][7 - r] = zmir(yb[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      v[1][r] = zdir(yb[r]);
      v[1][7 - r] = j0 == 0 ? zmir(yb[r]) : zmir(ya[r]);
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int jb = q == 0 ? jb0 : jb1;
    dft8<+1>(v[q]);
#pragma unroll
    for (int r = 0; r < 8; ++r) sm[(jb * 8 + r) * C + col] = v[q][r];
  }
  __syncthreads();
  col_pass_range<+1, LOGN, C, 1, S::NPASS - 1>(sm, a.tw, tid);
  if (PF) {
    cp_async_wait_all();
    __syncthreads();
  }

  // last pass straight to global: output r of butterfly jb is trace jb + r Ns;
  // real part -> column ta, imaginary part -> column ta + 1
  constexpr int Q = S::NPASS - 1, R = S::radix(Q), NB = 16 / R, Ns = S::ns(Q);
  float2 w[16];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = j0 + JS * q;
#pragma unroll
    for (int r = 0; r < R; ++r) w[q * R + r] = sm[(jb + r * (N / R)) * C + col];
  }
  float* out = a.out_real + slab * a.slab_real;
  const float* ew = a.ew ? a.ew + slab * a.slab_real : nullptr;
  const float* tm = a.tmask ? a.tmask + (slab / a.slabs_per_gather) * a.nx : nullptr;
  const bool vec = (a.nt & 1) == 0;
  float ss = 0.f;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = j0 + JS * q;
    if (Ns > 1) twiddle_r<R>(&w[q * R], base_twiddle<+1>(a.tw, S::tw_off(Q), jb));
    dft_r<+1, R>(&w[q * R]);
#pragma unroll
    for (int r = 0; r < (NXH ? R / 2 : R); ++r) {
      const int row = jb + r * Ns;
      if (row < a.nx && ta < a.nt) {
        const long long o = (long long)row * a.nt + ta;
        float2 x = w[q * R + r];
        const float g = tm ? __ldg(tm + row) : 1.f;
        if (vec && ta + 1 < a.nt) {
          float2 e = PF ? *(const float2*)(sew + row * 2 * C + 2 * col)
                        : (ew ? __ldg((const float2*)(ew + o)) : make_float2(1.f, 1.f));
          x.x *= g * e.x;
          x.y *= g * e.y;
          ss = fmaf(x.x, x.x, fmaf(x.y, x.y, ss));
          if (a.ew_sq) {
            x.x *= e.x;
            x.y *= e.y;
          }
          *(float2*)(out + o) = x;
        } else {
          const float ea = PF ? sew[row * 2 * C + 2 * col] : (ew ? __ldg(ew + o) : 1.f);
          const float xa = x.x * g * ea;
          out[o] = a.ew_sq ? xa * ea : xa;
          ss = fmaf(xa, xa, ss);
          if (ta + 1 < a.nt) {
            const float eb = PF ? sew[row * 2 * C + 2 * col + 1] : (ew ? __ldg(ew + o + 1) : 1.f);
            const float xb = x.y * g * eb;
            out[o + 1] = a.ew_sq ? xb * eb : xb;
            ss = fmaf(xb, xb, ss);
          }
        }
      }
    }
  }
  if (a.dot) block_accumulate((double)ss, a.dot + slab / a.slabs_per_gather);
}

template <int LOGN, int C>
cudaError_t launch_r2c_v(const XfftArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN, T = N * C / 16;
  const size_t smem = (size_t)N * C * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(xfft_r2c_kernel<LOGN, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(a.slabs, (a.nt + 2 * C - 1) / (2 * C));
  xfft_r2c_kernel<LOGN, C><<<grid, T, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN>
cudaError_t launch_r2c_tma(const XfftArgs& a, cudaStream_t s, bool* used) {
  constexpr int N = 1 << LOGN, C = 8, T = N * C / 16;
  *used = false;
  const long long slabs = a.slabs;
  R2cMaps mp;
  memset(&mp, 0, sizeof(mp));
  const int mode = a.cg_mode;
  if (!encode_tmap_f32_3d(&mp.in, a.in_real, a.nt, a.nx, slabs, 16, a.nx)) return cudaSuccess;
  if (mode && !encode_tmap_f32_3d(&mp.s, a.cg_s, a.nt, a.nx, slabs, 16, a.nx)) return cudaSuccess;
  if (mode == 1 && !encode_tmap_f32_3d(&mp.u, a.cg_u, a.nt, a.nx, slabs, 16, a.nx))
    return cudaSuccess;
  if (mode == 1 && a.cg_pout &&
      !encode_tmap_f32_3d(&mp.p2, a.cg_pout, a.nt, a.nx, slabs, 16, a.nx))
    return cudaSuccess;
  if (a.ew && !encode_tmap_f32_3d(&mp.w, a.ew, a.nt, a.nx, slabs, 16, a.nx)) return cudaSuccess;
  const bool p2r = mode == 1 && a.cg_p2_read;
  const bool urw = mode == 1 && a.cg_u_rw;
  if (p2r && (!a.cg_pout || !urw)) return cudaErrorInvalidValue;
  const int nslot = 1 + (mode ? 1 : 0) + (urw ? 1 : 0) + (p2r ? 1 : 0) + (a.ew ? 1 : 0);
  const size_t slot = ((size_t)a.nx * 64 + 127) & ~(size_t)127;
  const size_t smem = 128 + nslot * slot + (size_t)N * C * sizeof(float2) + 16;
  static int max_smem_set = 0;
  if ((int)smem > max_smem_set) {
    cudaError_t e = cudaFuncSetAttribute(xfft_r2c_tma<LOGN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    max_smem_set = (int)smem;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xfft_r2c_tma<LOGN>, T, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tt = (a.nt + 15) / 16;
  const long long n_tiles = slabs * n_tt;
  const long long grid = std::min<long long>(n_tiles, (long long)sms * per_sm);
  xfft_r2c_tma<LOGN><<<(unsigned)grid, T, smem, s>>>(a, mp, n_tt, n_tiles);
  *used = true;
  return cudaGetLastError();
}

template <int LOGN, int C, bool PF, bool NXH>
cudaError_t launch_c2r_k(const XfftArgs& a, cudaStream_t s, size_t smem) {
  constexpr int N = 1 << LOGN, T = N * C / 16;
  static size_t attr = 0;
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(xfft_c2r_kernel<LOGN, C, PF, NXH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  dim3 grid(a.slabs, (a.nt + 2 * C - 1) / (2 * C));
  xfft_c2r_kernel<LOGN, C, PF, NXH><<<grid, T, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, int C, bool PF>
cudaError_t launch_c2r_pf(const XfftArgs& a, cudaStream_t s, size_t smem) {
  return 2 * a.nx <= (1 << LOGN) ? launch_c2r_k<LOGN, C, PF, true>(a, s, smem)
                                 : launch_c2r_k<LOGN, C, PF, false>(a, s, smem);
}

// The weight tile goes through shared memory when there is a weight, its
// rows are 16-byte aligned (nt a multiple of 4) and the CTA's shared memory
// stays within 100 KB, so that two CTAs still fit on an SM (the register
// limit of the 512-thread CTAs); larger tiles would halve the occupancy.
template <int LOGN, int C>
cudaError_t launch_c2r_v(const XfftArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  const size_t base = (size_t)N * C * sizeof(float2);
  const size_t tile = (size_t)a.nx * 2 * C * sizeof(float);
  if (a.ew && (a.nt & 3) == 0 && base + tile <= 100 * 1024)
    return launch_c2r_pf<LOGN, C, true>(a, s, base + tile);
  return launch_c2r_pf<LOGN, C, false>(a, s, base);
}

// Column-tile variant: 16 complex columns per CTA (autotuner default) or 8;
// Nx >= 1024 always uses 8 (a CTA stays within 1024 threads and 64 KB).
template <int LOGN>
cudaError_t launch_r2c_t(const XfftArgs& a, cudaStream_t s) {
  if constexpr (LOGN <= 9) {
    if (a.cols == 16) return launch_r2c_v<LOGN, 16>(a, s);
  }
  return launch_r2c_v<LOGN, 8>(a, s);
}

template <int LOGN>
cudaError_t launch_c2r_t(const XfftArgs& a, cudaStream_t s) {
  if constexpr (LOGN <= 9) {
    if (a.cols == 16) return launch_c2r_v<LOGN, 16>(a, s);
  }
  return launch_c2r_v<LOGN, 8>(a, s);
}

}  // namespace

int xfft_log2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

cudaError_t launch_xfft_r2c(const XfftArgs& a, cudaStream_t s) {
  // the TMA kernel pays where the load streams several vectors (weights,
  // fused CGLS update); a plain transform keeps the wider non-TMA tile
  if (a.tma && (a.cg_mode || a.ew) && a.nx <= 256 && (a.nt & 3) == 0) {
    bool used = false;
    cudaError_t e = cudaSuccess;
    switch (xfft_log2(a.Nx)) {
      case 7: e = launch_r2c_tma<7>(a, s, &used); break;
      case 8: e = launch_r2c_tma<8>(a, s, &used); break;
      case 9: e = launch_r2c_tma<9>(a, s, &used); break;
      default: break;
    }
    if (e != cudaSuccess || used) return e;
  }
  switch (xfft_log2(a.Nx)) {
    case 4: return launch_r2c_t<4>(a, s);
    case 5: return launch_r2c_t<5>(a, s);
    case 6: return launch_r2c_t<6>(a, s);
    case 7: return launch_r2c_t<7>(a, s);
    case 8: return launch_r2c_t<8>(a, s);
    case 9: return launch_r2c_t<9>(a, s);
    case 10: return launch_r2c_t<10>(a, s);
    case 11: return launch_r2c_t<11>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_xfft_c2r(const XfftArgs& a, cudaStream_t s) {
  switch (xfft_log2(a.Nx)) {
    case 4: return launch_c2r_t<4>(a, s);
    case 5: return launch_c2r_t<5>(a, s);
    case 6: return launch_c2r_t<6>(a, s);
    case 7: return launch_c2r_t<7>(a, s);
    case 8: return launch_c2r_t<8>(a, s);
    case 9: return launch_c2r_t<9>(a, s);
    case 10: return launch_c2r_t<10>(a, s);
    case 11: return launch_c2r_t<11>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ashrt
