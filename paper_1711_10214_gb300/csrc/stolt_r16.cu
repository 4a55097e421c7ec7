// Radix-16 variant of the fused t-FFT + Stolt map row kernels (forward and
// adjoint of ch. 5 Eqs ch5_forward_operator / ch5_adj_operator, ch. 6 Eqs
// ch6_forward_operator / ch6_adj_operator), for Nt = 1024, 2048 and 4096.
//
// The operator, the tables (Stolt taps, adjoint sources, spectral weight, phase)
// and the CTA work split (one k_x row of a pair of gathers, the two rows
// interleaved as float4) are those of stolt_fwd.cu / stolt_adj.cu.  What
// changes is the transform: each thread holds 16 values instead of 8, so a
// length-Nt transform takes three Stockham passes (16 x 16 x {4, 8, 16})
// instead of four (8 x 8 x 8 x {2, 4}) and each element crosses shared memory
// two times fewer per transform.  The kernels are bound by shared-memory
// wavefronts, so this is the quantity that matters; the price is Nt/16
// threads per CTA with twice the registers each (the cap allows 168).
//
// Shared rows use the swizzle i ^ ((i >> 4) & 7) (float4 elements, eight per
// 128-byte bank row): the first pass writes 16 consecutive outputs per
// thread, i.e. a stride of 16 elements across the lanes, which this swizzle
// spreads over all eight 16-byte bank groups of every quarter warp.
#include <cuda_runtime.h>

#include "stolt_common.cuh"
#include "stolt_r16.cuh"

namespace ashrt {

namespace {

// Tensor-memory words of a thread (the forward's accumulated bins, the
// adjoint's twiddle powers) live in TMEM columns of the thread's own lane (a
// warp reaches only its quarter of the 128 lanes: warp w of a 128-thread CTA
// owns lanes 32w..32w+31).  Loads complete at tcgen05.wait::ld, which takes the loaded
// registers as operands so that no use is scheduled before it.
__device__ __forceinline__ void tm_ld16(uint32_t ta, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
}
__device__ __forceinline__ void tm_wait_ld(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
__device__ __forceinline__ void tm_st16(uint32_t ta, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};\n" ::"r"(ta),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tm_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all_but_1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

constexpr int kTmCols = 64;   // TMEM columns per CTA (power of two >= 32)

// 16 float2 values through 32 TMEM columns of the thread's lane.
__device__ __forceinline__ void tm_st_f2x16(uint32_t ta, const float2* v) {
  uint32_t r[16];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      r[2 * i] = __float_as_uint(v[8 * h + i].x);
      r[2 * i + 1] = __float_as_uint(v[8 * h + i].y);
    }
    tm_st16(ta + 16 * h, r);
  }
}
__device__ __forceinline__ void tm_ld_f2x16(uint32_t ta, float2* v) {
  uint32_t r0[16], r1[16];
  tm_ld16(ta, r0);
  tm_ld16(ta + 16, r1);
  tm_wait_ld(r0);
  tm_wait_ld(r1);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = make_float2(__uint_as_float(r0[2 * i]), __uint_as_float(r0[2 * i + 1]));
    v[8 + i] = make_float2(__uint_as_float(r1[2 * i]), __uint_as_float(r1[2 * i + 1]));
  }
}

// Resident CTAs per SM each length is compiled for (register cap 65536 /
// (threads x CTAs)): Nt 1024 -> 64 threads x 6, 2048 -> 128 x 3, 4096 -> 256 x 1
// (the last is bound by shared memory to one CTA anyway).
template <int LOGN>
constexpr int r16_minb() {
  return LOGN == 10 ? 6 : (LOGN == 11 ? 3 : 1);
}

// Forward rows: as stolt_fwd_rows, with 16 bins per thread.  HALF: nt <=
// Nt / 2, so the staged panel fills only the first half of each transform
// (inputs tid + r Nt/16 with r >= 8 are zero padding).
template <int LOGN, bool SHIFT, bool HALF>
__global__ void __launch_bounds__((1 << LOGN) / 16, r16_minb<LOGN>())
stolt_fwd_rows16(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 16;
  using S = Sched16<LOGN>;
  extern __shared__ float4 smem4[];
  float4* buf = smem4;                          // N interleaved (A, B) values
  float2* stage = (float2*)(smem4 + N);         // next panel: row A [ld], row B [ld]
  unsigned* stap0 = (unsigned*)(stage + 2 * a.ld);
  unsigned* stap1 = stap0 + a.taps_ld;
  const int tid = threadIdx.x, l = blockIdx.x, b0 = 2 * blockIdx.y;
  const bool hasB = b0 + 1 < a.batch;
  const float2* xA = a.X + (long long)b0 * a.x_batch + (long long)l * a.ld;
  const float2* xB = hasB ? xA + a.x_batch : nullptr;

  float4 acc[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  const unsigned* trow = a.taps + (long long)l * a.taps_ld;
  const long long tstep = (long long)a.Lh * a.taps_ld;
  stage_rows(stage, xA, xB, a.ld, tid, T);
  stage_taps(stap0, trow, a.taps_ld, tid, T);
  cp_async_commit();

  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    const unsigned* stap = (p & 1) ? stap1 : stap0;
    cp_async_wait_all();
    __syncthreads();
    float4 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = tid + r * T;
      if (HALF && r >= 8) {
        v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      const float2 za = i < a.nt ? stage[i] : make_float2(0.f, 0.f);
      const float2 zb = (hasB && i < a.nt) ? stage[a.ld + i] : make_float2(0.f, 0.f);
      v[r] = pack2(za, zb);
    }
    __syncthreads();
    if (p + 1 < a.P) {
      const long long o = (long long)(p + 1) * a.x_panel;
      const int ivn = iv + 1 == a.nv ? 0 : iv + 1;
      stage_rows(stage, xA + o, hasB ? xB + o : nullptr, a.ld, tid, T);
      stage_taps((p & 1) ? stap0 : stap1, trow + ivn * tstep, a.taps_ld, tid, T);
      cp_async_commit();
    }
    r16_first_pass<-1, float4, HALF>(buf, v, tid);
    r16_pass_range<-1, LOGN, 1, S::NPASS, float4, true>(buf, a.tw16, tid);   // natural, unswizzled

#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int k = tid + T * s;
      const bool pos = s < 8;                      // k < N/2 exactly for the first half of s
      const Tap t = tap_decode_side<N>(k, stap[pos ? k : N - k], pos);
      if (t.valid) {
        float4 vk = cscale(buf[t.i0], t.w0);
        vk = cfma(t.w1, buf[t.i1], vk);
        if (SHIFT) vk = cmul(vk, __ldg(a.phase + (long long)jt * N + k));
        acc[s] = cadd(acc[s], vk);
      }
    }
    if (++iv == a.nv) {
      iv = 0;
      ++jt;
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 16; ++s) acc[s] = cscale(acc[s], __ldg(a.wt + tid + T * s));
  r16_first_pass<+1>(buf, acc, tid);
  r16_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw16, tid);
  float2* yA = a.Yw + (long long)b0 * a.y_batch + (long long)l * a.ld;
  r16_last_pass_global<+1, LOGN, float4, HALF>(buf, a.tw16, tid, yA,
                                               hasB ? yA + a.y_batch : nullptr, a.nt);
}

// Adjoint rows: as stolt_adj_rows (gather form of the transposed map over the
// source table), with 16 output bins per thread.
template <int LOGN, bool SHIFT, bool HALF>
__global__ void __launch_bounds__((1 << LOGN) / 16, r16_minb<LOGN>())
stolt_adj_rows16(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 16, H = N / 2;
  using S = Sched16<LOGN>;
  extern __shared__ float4 smem4[];
  float4* buf = smem4;                          // per-panel w_tau spectrum, then its inverse FFT
  float4* dsp = smem4 + N;                      // data spectrum x W (both gathers)
  uint2* stab = (uint2*)(smem4 + 2 * N);        // source-table row of the current panel
  uint32_t* tslot = (uint32_t*)(stab + a.atab_ld);
  const int tid = threadIdx.x, l = blockIdx.x, b0 = 2 * blockIdx.y;
  const bool hasB = b0 + 1 < a.batch;
  const float2* yA = a.Y + (long long)b0 * a.y_batch + (long long)l * a.ld;
  const float2* yB = hasB ? yA + a.y_batch : nullptr;
  const uint2* arow = a.atab + (long long)l * a.atab_ld;
  const long long astep = (long long)a.Lh * a.atab_ld;
  stage_tab(stab, arow, a.atab_ld, tid, T);
  cp_async_commit();

  // Nt = 2048 (128 threads, one per TMEM lane): the inverse transform's
  // twiddle powers depend on the thread and the pass, not on the panel.  They
  // are formed once (by the products the passes would form) and kept in 64
  // TMEM columns of the thread's lane: columns 0..31 the radix-16 pass's
  // w^1..w^15, 32..63 the last pass's w^1..w^7 of its two butterflies.
  constexpr bool TMT = LOGN == 11;
  uint32_t tpw = 0;
  if constexpr (TMT) {
    const int warp = tid >> 5;
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                       (unsigned)__cvta_generic_to_shared(tslot)),
                   "r"((uint32_t)kTmCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    tpw = *tslot + ((uint32_t)(32 * warp) << 16);
    float2 pw[16];
    pw[0] = make_float2(0.f, 0.f);
    twiddle_powers<16>(base_twiddle<+1>(a.tw16, S::tw_off(1), tid & 15), pw);
    tm_st_f2x16(tpw, pw);
    pw[8] = make_float2(0.f, 0.f);
    twiddle_powers<8>(base_twiddle<+1>(a.tw16, S::tw_off(2), tid), pw);
    twiddle_powers<8>(base_twiddle<+1>(a.tw16, S::tw_off(2), tid + T), pw + 8);
    tm_st_f2x16(tpw + 32, pw);
    tm_wait_st();
  }

  {
    float4 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = tid + r * T;
      const float2 za = i < a.nt ? __ldg(yA + i) : make_float2(0.f, 0.f);
      const float2 zb = (yB && i < a.nt) ? __ldg(yB + i) : make_float2(0.f, 0.f);
      v[r] = pack2(za, zb);
    }
    r16_first_pass<-1>(buf, v, tid);
  }
  r16_pass_range<-1, LOGN, 1, S::NPASS, float4, true>(buf, a.tw16, tid);
  // With asymptote shifts the data spectrum is kept multiplied by the
  // conjugate phase of the current shift (shift 0 here, then moved on each
  // time the shift changes), so the gathers need no per-source phase.
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int k = tid + T * s;
    float4 dk = cscale(buf[k], __ldg(a.wt + k));   // natural order, unswizzled
    if (SHIFT) dk = cmul(dk, cconj(__ldg(a.phase + k)));
    dsp[k] = dk;
  }

  float2* xA = a.Xw + (long long)b0 * a.x_batch + (long long)l * a.ld;
  float2* xB = hasB ? xA + a.x_batch : nullptr;
  int iv = 0, jt = 0;
  int km = __ldg(a.kmin + l);                   // cone start of the panel's (velocity, k_x)
  for (int p = 0; p < a.P; ++p) {
    cp_async_wait_all();
    __syncthreads();
    if (SHIFT && iv == 0 && p > 0) {
      // shift jt - 1 -> jt: each thread moves the bins it wrote, after every
      // gather of the previous panel (the barrier above) and before the next
      const float2* ph1 = a.phase + (long long)jt * N;
      const float2* ph0 = ph1 - N;
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        const int k = tid + T * s;
        dsp[k] = cmul(dsp[k], cmul(cconj(__ldg(ph1 + k)), __ldg(ph0 + k)));
      }
      __syncthreads();
    }
    const bool mapped = km < H;
    // the next panel's, loaded a panel ahead of its use
    if (p + 1 < a.P) km = __ldg(a.kmin + (iv + 1 == a.nv ? 0 : iv + 1) * a.Lh + l);
    float4 accs[16];
#pragma unroll
    for (int s = 0; s < 16; ++s)
      accs[s] = mapped ? adj_gather_bin<N, 0, false>(dsp, stab, tid + T * s, nullptr, s < 8)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0 && mapped) accs[0] = adj_gather_bin0_mirror<N, 0, false>(dsp, stab, nullptr, accs[0]);
    // its barrier also ends every thread's reads of the source-table row
    r16_first_pass<+1>(buf, accs, tid);
    if (p + 1 < a.P) {
      const int ivn = iv + 1 == a.nv ? 0 : iv + 1;
      stage_tab(stab, arow + ivn * astep, a.atab_ld, tid, T);
      cp_async_commit();
    }
    const long long o = (long long)p * a.x_panel;
    if constexpr (TMT) {
      static_assert(S::NPASS == 3 && S::radix(1) == 16 && S::radix(2) == 8, "Nt 2048 schedule");
      float2 pw[16];
      tm_ld_f2x16(tpw, pw);
      r16_pass<+1, N, 16, float4, false, true>(buf, S::ns(1), a.tw16, S::tw_off(1), tid, pw);
      tm_ld_f2x16(tpw + 32, pw);
      r16_last_pass_global<+1, LOGN, float4, HALF, true>(buf, a.tw16, tid, xA + o,
                                                         xB ? xB + o : nullptr, a.nt, pw);
    } else {
      r16_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw16, tid);
      r16_last_pass_global<+1, LOGN, float4, HALF>(buf, a.tw16, tid, xA + o,
                                                   xB ? xB + o : nullptr, a.nt);
    }
    if (++iv == a.nv) {
      iv = 0;
      ++jt;
    }
  }
  if constexpr (TMT) {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if ((tid >> 5) == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(*tslot),
                   "r"((uint32_t)kTmCols));
    }
  }
}


// Forward rows for Nt = 2048 with the accumulator in tensor memory: as
// stolt_fwd_rows16<11>, but each thread's 16 accumulated bins live in TMEM
// instead of 64 registers, and the tap row is single-buffered (staged at the
// start of a panel, waited for before its map), so that 128 registers and
// 53 KB of shared memory per CTA let four CTAs share an SM instead of three:
// the kernel is issue-bound and hides its shared-memory latency with the extra
// warps.  TMEM per CTA: 128 columns, the sums in 0..63 and the twiddle powers
// of the thread's butterflies (they depend on the thread and the pass, not on
// the panel: formed once, by the products the passes would form) in 64..127;
// four CTAs, the most that fit an SM, hold its 512 columns.  With asymptote
// shifts (panels p = j nv + i) the sums are kept in the phase frame of the
// current shift j, S_j = sum_{j' <= j} (phi_j' / phi_j) A_j', A_j' the
// unphased sum over shift j''s velocities and phi_j = exp(-i w tau0_j): each
// panel adds its map without a phase, the sums turn by phi_{j-1} conj(phi_j)
// when j changes, and by phi_{last} at the end.  cp.async groups, in commit order: rows of panel p (issued
// during panel p - 1), taps of panel p (issued after panel p's first barrier,
// which ends every read of panel p - 1), rows of p + 1 (a group may be
// empty): a panel starts once all have landed, and its map once all but the
// newest have (the wait rides on the last transform pass's closing barrier).
template <bool SHIFT, bool HALF>
__global__ void __launch_bounds__(128, 4) stolt_fwd_rows16_tm(RowArgs a) {
  constexpr int LOGN = 11, N = 1 << LOGN, T = N / 16;
  using S = Sched16<LOGN>;
  extern __shared__ float4 smem4[];
  float4* buf = smem4;                          // N interleaved (A, B) values
  float2* stage = (float2*)(smem4 + N);         // next panel: row A [ld], row B [ld]
  unsigned* stap = (unsigned*)(stage + 2 * a.ld);
  uint32_t* tslot = (uint32_t*)(stap + a.taps_ld);
  const int tid = threadIdx.x, warp = tid >> 5, l = blockIdx.x, b0 = 2 * blockIdx.y;
  const bool hasB = b0 + 1 < a.batch;
  const float2* xA = a.X + (long long)b0 * a.x_batch + (long long)l * a.ld;
  const float2* xB = hasB ? xA + a.x_batch : nullptr;
  const unsigned* trow = a.taps + (long long)l * a.taps_ld;
  const long long tstep = (long long)a.Lh * a.taps_ld;
  stage_rows(stage, xA, xB, a.ld, tid, T);
  cp_async_commit();

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(tslot)),
                 "r"((uint32_t)(2 * kTmCols)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tacc = *tslot + ((uint32_t)(32 * warp) << 16);
  const uint32_t tpw = tacc + kTmCols;
  {
    uint32_t z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0u;
#pragma unroll
    for (int c = 0; c < 4; ++c) tm_st16(tacc + 16 * c, z);
    static_assert(S::NPASS == 3 && S::radix(1) == 16 && S::radix(2) == 8, "Nt 2048 schedule");
    float2 pw[16];
    pw[0] = make_float2(0.f, 0.f);
    twiddle_powers<16>(base_twiddle<-1>(a.tw16, S::tw_off(1), tid & 15), pw);
    tm_st_f2x16(tpw, pw);
    pw[8] = make_float2(0.f, 0.f);
    twiddle_powers<8>(base_twiddle<-1>(a.tw16, S::tw_off(2), tid), pw);
    twiddle_powers<8>(base_twiddle<-1>(a.tw16, S::tw_off(2), tid + T), pw + 8);
    tm_st_f2x16(tpw + 32, pw);
  }

  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    // rows of panel p landed; every read of the previous panel (its map's
    // reads of buf and of the tap row) is done, so its tap row is restaged
    cp_async_wait_all();
    __syncthreads();
    stage_taps(stap, trow + iv * tstep, a.taps_ld, tid, T);
    cp_async_commit();
    float4 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = tid + r * T;
      if (HALF && r >= 8) {
        v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      const float2 za = i < a.nt ? stage[i] : make_float2(0.f, 0.f);
      const float2 zb = (hasB && i < a.nt) ? stage[a.ld + i] : make_float2(0.f, 0.f);
      v[r] = pack2(za, zb);
    }
    // its barrier also ends every thread's reads of the staged rows, which
    // are then restaged with the next panel's
    r16_first_pass<-1, float4, HALF>(buf, v, tid);
    if (p + 1 < a.P) {
      const long long o = (long long)(p + 1) * a.x_panel;
      stage_rows(stage, xA + o, hasB ? xB + o : nullptr, a.ld, tid, T);
    }
    cp_async_commit();
    {
      tm_wait_st();                             // the powers (and the zeroed sums) are stored
      float2 pw[16];
      tm_ld_f2x16(tpw, pw);
      r16_pass<-1, N, 16, float4, false, true>(buf, S::ns(1), a.tw16, S::tw_off(1), tid, pw);
      tm_ld_f2x16(tpw + 32, pw);
      // the last pass leaves its natural-order output unswizzled; before its
      // closing barrier the tap row of panel p (every cp.async group but the
      // newest, the rows of panel p + 1) has landed
      r16_pass<-1, N, 8, float4, true, true, true>(buf, S::ns(2), a.tw16, S::tw_off(2), tid, pw);
    }
    tm_wait_st();                               // the previous panel's sums are in TMEM
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t r[16];
      tm_ld16(tacc + 16 * c, r);
      float4 vk[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int s = 4 * c + j, k = tid + T * s;
        const bool pos = s < 8;                    // k < N/2 exactly for the first half of s
        const Tap t = tap_decode_side<N>(k, stap[pos ? k : N - k], pos);
        vk[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t.valid) {
          vk[j] = cscale(buf[t.i0], t.w0);
          vk[j] = cfma(t.w1, buf[t.i1], vk[j]);
        }
      }
      tm_wait_ld(r);
      if (SHIFT && iv == 0 && p > 0) {
        // shift jt - 1 -> jt: the sums move to the new shift's phase frame
        const float2* ph1 = a.phase + (long long)jt * N;
        const float2* ph0 = ph1 - N;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = tid + T * (4 * c + j);
          float4 sk = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                  __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
          sk = cmul(sk, cmul(__ldg(ph0 + k), cconj(__ldg(ph1 + k))));
          r[4 * j] = __float_as_uint(sk.x);
          r[4 * j + 1] = __float_as_uint(sk.y);
          r[4 * j + 2] = __float_as_uint(sk.z);
          r[4 * j + 3] = __float_as_uint(sk.w);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        r[4 * j] = __float_as_uint(__uint_as_float(r[4 * j]) + vk[j].x);
        r[4 * j + 1] = __float_as_uint(__uint_as_float(r[4 * j + 1]) + vk[j].y);
        r[4 * j + 2] = __float_as_uint(__uint_as_float(r[4 * j + 2]) + vk[j].z);
        r[4 * j + 3] = __float_as_uint(__uint_as_float(r[4 * j + 3]) + vk[j].w);
      }
      tm_st16(tacc + 16 * c, r);
    }
    if (++iv == a.nv) {
      iv = 0;
      ++jt;
    }
  }
  tm_wait_st();
  float4 acc[16];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t r[16];
    tm_ld16(tacc + 16 * c, r);
    tm_wait_ld(r);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      acc[4 * c + j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                   __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(*tslot),
                 "r"((uint32_t)(2 * kTmCols)));
  }
  // with asymptote shifts the sums are in the last shift's phase frame
  const float2* phl = SHIFT ? a.phase + (long long)(a.nt0 - 1) * N : nullptr;
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int k = tid + T * s;
    if (SHIFT) acc[s] = cmul(acc[s], __ldg(phl + k));
    acc[s] = cscale(acc[s], __ldg(a.wt + k));
  }
  r16_first_pass<+1>(buf, acc, tid);
  r16_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw16, tid);
  float2* yA = a.Yw + (long long)b0 * a.y_batch + (long long)l * a.ld;
  r16_last_pass_global<+1, LOGN, float4, HALF>(buf, a.tw16, tid, yA,
                                               hasB ? yA + a.y_batch : nullptr, a.nt);
}

template <bool SHIFT, bool HALF>
cudaError_t launch_fwd16_tm_h(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << 11;
  static bool attr = false;
  const size_t smem = (size_t)N * sizeof(float4) + (size_t)2 * a.ld * sizeof(float2) +
                      (size_t)a.taps_ld * sizeof(unsigned) + 16;
  cudaError_t e = set_smem(stolt_fwd_rows16_tm<SHIFT, HALF>, smem_cap<11>(true), attr);
  if (e != cudaSuccess) return e;
  stolt_fwd_rows16_tm<SHIFT, HALF><<<dim3(a.Lh, (a.batch + 1) / 2), N / 16, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, bool SHIFT, bool HALF>
cudaError_t launch_fwd16_h(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)N * sizeof(float4) + (size_t)2 * a.ld * sizeof(float2) +
                      (size_t)2 * a.taps_ld * sizeof(unsigned);
  cudaError_t e = set_smem(stolt_fwd_rows16<LOGN, SHIFT, HALF>, smem_cap<LOGN>(true), attr);
  if (e != cudaSuccess) return e;
  stolt_fwd_rows16<LOGN, SHIFT, HALF><<<dim3(a.Lh, (a.batch + 1) / 2), N / 16, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, bool SHIFT>
cudaError_t launch_fwd16(const RowArgs& a, cudaStream_t s) {
  return 2 * a.nt <= a.Nt ? launch_fwd16_h<LOGN, SHIFT, true>(a, s)
                          : launch_fwd16_h<LOGN, SHIFT, false>(a, s);
}

template <int LOGN, bool SHIFT, bool HALF>
cudaError_t launch_adj16_h(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)2 * N * sizeof(float4) + (size_t)a.atab_ld * sizeof(uint2) + 16;
  cudaError_t e = set_smem(stolt_adj_rows16<LOGN, SHIFT, HALF>, smem_cap<LOGN>(false) + 16, attr);
  if (e != cudaSuccess) return e;
  stolt_adj_rows16<LOGN, SHIFT, HALF><<<dim3(a.Lh, (a.batch + 1) / 2), N / 16, smem, s>>>(a);
  return cudaGetLastError();
}

// HALF: nt <= Nt / 2, so each panel's inverse transform keeps only its
// lower half and the last pass forms only those outputs.
template <int LOGN, bool SHIFT>
cudaError_t launch_adj16(const RowArgs& a, cudaStream_t s) {
  return 2 * a.nt <= a.Nt ? launch_adj16_h<LOGN, SHIFT, true>(a, s)
                          : launch_adj16_h<LOGN, SHIFT, false>(a, s);
}

}  // namespace

bool rows16_supported(int logNt) { return logNt >= 10 && logNt <= 12; }

cudaError_t launch_stolt_fwd_rows16(const RowArgs& a, cudaStream_t s) {
  if (!a.tw16) return cudaErrorInvalidValue;
  const bool sh = a.phase != nullptr;
  switch (row_log2(a.Nt)) {
    case 10: return sh ? launch_fwd16<10, true>(a, s) : launch_fwd16<10, false>(a, s);
    case 11: return sh ? launch_fwd16<11, true>(a, s) : launch_fwd16<11, false>(a, s);
    case 12: return sh ? launch_fwd16<12, true>(a, s) : launch_fwd16<12, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

// The tensor-memory forward (Nt = 2048 only; other lengths take the register form).
cudaError_t launch_stolt_fwd_rows16_tm(const RowArgs& a, cudaStream_t s) {
  if (!a.tw16) return cudaErrorInvalidValue;
  if (row_log2(a.Nt) != 11) return launch_stolt_fwd_rows16(a, s);
  const bool sh = a.phase != nullptr, half = 2 * a.nt <= a.Nt;
  if (sh) return half ? launch_fwd16_tm_h<true, true>(a, s) : launch_fwd16_tm_h<true, false>(a, s);
  return half ? launch_fwd16_tm_h<false, true>(a, s) : launch_fwd16_tm_h<false, false>(a, s);
}

cudaError_t launch_stolt_adj_rows16(const RowArgs& a, cudaStream_t s) {
  if (!a.tw16) return cudaErrorInvalidValue;
  const bool sh = a.phase != nullptr;
  switch (row_log2(a.Nt)) {
    case 10: return sh ? launch_adj16<10, true>(a, s) : launch_adj16<10, false>(a, s);
    case 11: return sh ? launch_adj16<11, true>(a, s) : launch_adj16<11, false>(a, s);
    case 12: return sh ? launch_adj16<12, true>(a, s) : launch_adj16<12, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ashrt
