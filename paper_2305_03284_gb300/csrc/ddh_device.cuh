// Device building blocks of the DDH-MBIR frame step (sm_103a, FP32, complex64).
//
//  * complex helpers and radix-2/4/8 DFT butterflies;
//  * a warp-per-row Stockham FFT held in shared memory (mixed radix 8/4), used for every
//    1-D pass of the unitary 2-D DFT F of Sec. 2;
//  * per-pixel arithmetic: angle wrap, aperture test, q-GGMRF surrogate weight, and the
//    ICD pixel update (root of W r^3 - C r^2 + r - s = 0 minimising the 1-D surrogate);
//  * TMA (cp.async.bulk) and mbarrier wrappers with bounded waits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ddh {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kInvTwoPi = 0.15915494309189533577f;
// 8-neighbour weights summing to one (orthogonal 1/(4 + 2 sqrt 2), diagonal that / sqrt 2)
constexpr float kBnn = 0.14644660940672624f;
constexpr float kBdiag = 0.10355339059327377f;

// ------------------------------------------------------------------------------------ complex
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float c_abs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
// a * (S i): S = -1 multiplies by -i, S = +1 by +i
template <int S>
__device__ __forceinline__ float2 c_mul_si(float2 a) {
  return S < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ------------------------------------------------------------------------------ DFT kernels
// y_q = sum_m x_m exp(S 2 pi i m q / R), in place; S = -1 forward, +1 inverse (unscaled).
template <int S>
__device__ __forceinline__ void dft2(float2* x) {
  const float2 t = x[0];
  x[0] = c_add(t, x[1]);
  x[1] = c_sub(t, x[1]);
}

template <int S>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 a0 = c_add(x0, x2), a1 = c_sub(x0, x2);
  const float2 b0 = c_add(x1, x3), b1 = c_mul_si<S>(c_sub(x1, x3));
  x0 = c_add(a0, b0);
  x2 = c_sub(a0, b0);
  x1 = c_add(a1, b1);
  x3 = c_sub(a1, b1);
}

template <int S>
__device__ __forceinline__ void dft4(float2* x) { dft4<S>(x[0], x[1], x[2], x[3]); }

template <int S>
__device__ __forceinline__ void dft8(float2* x) {
  float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<S>(e0, e1, e2, e3);
  dft4<S>(o0, o1, o2, o3);
  const float h = 0.70710678118654752440f;
  // twiddles exp(S 2 pi i q / 8), q = 1, 2, 3
  o1 = c_mul(o1, make_float2(h, S * h));
  o2 = c_mul_si<S>(o2);
  o3 = c_mul(o3, make_float2(-h, S * h));
  x[0] = c_add(e0, o0); x[4] = c_sub(e0, o0);
  x[1] = c_add(e1, o1); x[5] = c_sub(e1, o1);
  x[2] = c_add(e2, o2); x[6] = c_sub(e2, o2);
  x[3] = c_add(e3, o3); x[7] = c_sub(e3, o3);
}

template <int R, int S>
__device__ __forceinline__ void dft_r(float2* x) {
  if constexpr (R == 2) dft2<S>(x);
  else if constexpr (R == 4) dft4<S>(x);
  else dft8<S>(x);
}

// Shared-memory placement of element i of a row: the low four bits are XORed with the next
// four, so that the strided stores of the early Stockham passes (stride 4 or 32 elements)
// spread over all banks.  Every reader and writer of a row buffer uses this placement.
__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 4) & 15); }

// ------------------------------------------------------------------------------- row FFT
// One Stockham radix-R pass over a length-N row owned by one warp (element e at row[swz(e)]).
// Group i (0 <= i < N/R) reads x_m = element i + m N/R, multiplies by exp(S 2 pi i m k /(P R)) with k = i mod P, takes
// the R-point DFT and writes y_q to element (i - k) R + k + q P.  All reads of the warp finish
// before any write, so the pass runs in place.  `tw[t] = exp(-2 pi i t / N)`.
// Reads element e of a swizzled row.
struct RowLoad {
  const float2* row;
  __device__ __forceinline__ float2 operator()(int e) const { return row[swz(e)]; }
};

// `load(e)` supplies element e of the input (the row itself, or another buffer for a first
// pass that gathers its input); the output always goes to `row`.
template <int N, int R, int P, int S, typename Load>
__device__ __forceinline__ void stockham_pass(float2* row, const float2* __restrict__ tw, int lane, const Load& load) {
  constexpr int G = N / R;
  constexpr int GPL = (G + 31) / 32;
  float2 v[GPL][R];
#pragma unroll
  for (int g = 0; g < GPL; ++g) {
    const int i = lane + 32 * g;
    if (G % 32 == 0 || i < G) {
#pragma unroll
      for (int m = 0; m < R; ++m) v[g][m] = load(i + m * G);
    }
  }
  __syncwarp();
#pragma unroll
  for (int g = 0; g < GPL; ++g) {
    const int i = lane + 32 * g;
    if (G % 32 == 0 || i < G) {
      const int k = i & (P - 1);
      if constexpr (P > 1) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          float2 w = tw[(m * k) * (N / (P * R))];
          if constexpr (S > 0) w.y = -w.y;
          v[g][m] = c_mul(v[g][m], w);
        }
      }
      dft_r<R, S>(v[g]);
      const int j = (i - k) * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) row[swz(j + q * P)] = v[g][q];
    }
  }
  __syncwarp();
}

// Radix schedules of the length-N row DFT (the autotuner picks one per N; every schedule is
// the same DFT, up to rounding).
template <int N>
struct FftSchedules;
template <>
struct FftSchedules<32> { static constexpr int count = 2; };
template <>
struct FftSchedules<64> { static constexpr int count = 2; };
template <>
struct FftSchedules<128> { static constexpr int count = 2; };
template <>
struct FftSchedules<256> { static constexpr int count = 3; };
template <>
struct FftSchedules<512> { static constexpr int count = 1; };

// Unscaled length-N DFT of one shared-memory row by one warp (S = -1 forward, +1 inverse),
// radix schedule V:  32: {8,4} | {4,8};  64: {8,8} | {4,4,4};  128: {8,4,4} | {2,8,8};
// 256: {8,8,4} | {4,4,4,4} | {4,8,8};  512: {8,8,8}.  The first pass takes its input from
// `first(e)` (a gather from another buffer, or the row itself), the later ones from the row.
template <int N, int S, int V, typename Load>
__device__ __forceinline__ void fft_row_from(float2* row, const float2* __restrict__ tw, int lane, const Load& first) {
  const RowLoad rl{row};
  static_assert(N == 32 || N == 64 || N == 128 || N == 256 || N == 512, "unsupported N");
  static_assert(V >= 0 && V < FftSchedules<N>::count, "unknown schedule");
  if constexpr (N == 32) {
    if constexpr (V == 0) {
      stockham_pass<32, 8, 1, S>(row, tw, lane, first);
      stockham_pass<32, 4, 8, S>(row, tw, lane, rl);
    } else {
      stockham_pass<32, 4, 1, S>(row, tw, lane, first);
      stockham_pass<32, 8, 4, S>(row, tw, lane, rl);
    }
  } else if constexpr (N == 64) {
    if constexpr (V == 0) {
      stockham_pass<64, 8, 1, S>(row, tw, lane, first);
      stockham_pass<64, 8, 8, S>(row, tw, lane, rl);
    } else {
      stockham_pass<64, 4, 1, S>(row, tw, lane, first);
      stockham_pass<64, 4, 4, S>(row, tw, lane, rl);
      stockham_pass<64, 4, 16, S>(row, tw, lane, rl);
    }
  } else if constexpr (N == 128) {
    if constexpr (V == 0) {
      stockham_pass<128, 8, 1, S>(row, tw, lane, first);
      stockham_pass<128, 4, 8, S>(row, tw, lane, rl);
      stockham_pass<128, 4, 32, S>(row, tw, lane, rl);
    } else {
      stockham_pass<128, 2, 1, S>(row, tw, lane, first);
      stockham_pass<128, 8, 2, S>(row, tw, lane, rl);
      stockham_pass<128, 8, 16, S>(row, tw, lane, rl);
    }
  } else if constexpr (N == 256) {
    if constexpr (V == 0) {
      stockham_pass<256, 8, 1, S>(row, tw, lane, first);
      stockham_pass<256, 8, 8, S>(row, tw, lane, rl);
      stockham_pass<256, 4, 64, S>(row, tw, lane, rl);
    } else if constexpr (V == 1) {
      stockham_pass<256, 4, 1, S>(row, tw, lane, first);
      stockham_pass<256, 4, 4, S>(row, tw, lane, rl);
      stockham_pass<256, 4, 16, S>(row, tw, lane, rl);
      stockham_pass<256, 4, 64, S>(row, tw, lane, rl);
    } else {
      stockham_pass<256, 4, 1, S>(row, tw, lane, first);
      stockham_pass<256, 8, 4, S>(row, tw, lane, rl);
      stockham_pass<256, 8, 32, S>(row, tw, lane, rl);
    }
  } else {
    stockham_pass<512, 8, 1, S>(row, tw, lane, first);
    stockham_pass<512, 8, 8, S>(row, tw, lane, rl);
    stockham_pass<512, 8, 64, S>(row, tw, lane, rl);
  }
}

// Row DFT in place (the first pass reads the row itself).
template <int N, int S, int V = 0>
__device__ __forceinline__ void fft_row(float2* row, const float2* __restrict__ tw, int lane) {
  fft_row_from<N, S, V>(row, tw, lane, RowLoad{row});
}

// ------------------------------------------------------------------------ warp reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------- pixel math
// Angle into (-pi, pi].
__device__ __forceinline__ float wrap_pi(float d) {
  d = fmaf(-kTwoPi, rintf(d * kInvTwoPi), d);
  if (d > kPi) d -= kTwoPi;
  else if (d <= -kPi) d += kTwoPi;
  return d;
}

// Pixel (row, col) lies in the pupil disc of diameter d centred at ((N-1)/2, (N-1)/2):
// (2 col - (N-1))^2 + (2 row - (N-1))^2 <= d^2, evaluated exactly in integers
// (`ap_lim` = floor(d^2)).
__device__ __forceinline__ int ap_dist2(int v, int n) { const int t = 2 * v - (n - 1); return t * t; }

// Tile (T, X) of the G x G tile grid (G = 2^gs) holds a pupil pixel: the tile's smallest
// squared distances along y and along x together (the test is separable and exact).
__device__ __forceinline__ bool tile_in_pupil(int T, int X, int gs, int n, int ap_lim) {
  int my = 1 << 30, mx = 1 << 30;
  for (int j = 0; j < (1 << gs); ++j) {
    my = min(my, ap_dist2((T << gs) + j, n));
    mx = min(mx, ap_dist2((X << gs) + j, n));
  }
  return my + mx <= ap_lim;
}

// q-GGMRF surrogate weight rho'(D)/D for q = 2:
//   (T sigma)^(p-2) sigma^(-p) (q/p + u) / (1 + u)^2,  u = (|D| / (T sigma))^(q - p).
__device__ __forceinline__ float prior_weight(float delta, float w0, float inv_tsig, float q_minus_p,
                                              float q_over_p) {
  const float t = fabsf(delta) * inv_tsig;
  const float u = t > 0.f ? powf(t, q_minus_p) : 0.f;
  const float d = 1.f + u;
  return w0 * (q_over_p + u) / (d * d);
}

// Hardware approximations (PTX ex2.approx / rcp.approx: a few ulp) used where the result
// feeds a quantity compared against FP64 at 2e-5.
__device__ __forceinline__ float hw_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// log2 on the MUFU unit, subnormal inputs flushed to zero (log2 -> -inf).
__device__ __forceinline__ float hw_log2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float hw_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Same weight with the power taken through the hardware log2 / exp2 and one reciprocal
// (relative error of the weight a few 1e-7, far inside the step's FP32-vs-FP64 tolerance).
__device__ __forceinline__ float prior_weight_fast(float delta, float w0, float inv_tsig, float q_minus_p,
                                                   float q_over_p) {
  const float t = fabsf(delta) * inv_tsig;
  const float u = t > 0.f ? hw_exp2(q_minus_p * hw_log2(t)) : 0.f;
  const float d = 1.f + u;
  return (w0 * (q_over_p + u)) * hw_rcp(d * d);
}

// ICD pixel update: the positive real root of f(r) = W r^3 - C r^2 + r - s minimising
// h(r) = log r + s/r + W r^2/2 - C r (ties: the smaller root); r = s when W = 0.
// Closed form on the depressed cubic t^3 + P t + Q (r = t + C/(3W)): trigonometric form
// for three real roots, hyperbolic forms for one; then two Newton steps on f.
__device__ __forceinline__ float newton_cubic(float r, float W, float C, float s) {
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float f = fmaf(fmaf(fmaf(W, r, -C), r, 1.f), r, -s);
    const float fp = fmaf(fmaf(3.f * W, r, -2.f * C), r, 1.f);
    const float rn = r - f / fp;
    if (fp != 0.f && isfinite(rn) && rn > 0.f) r = rn;
  }
  return r;
}

__device__ __forceinline__ float icd_root(float W, float C, float s) {
  if (!(W > 0.f)) return s;
  const float iw = 1.f / W;
  const float shift = C * iw * (1.f / 3.f);                     // -a/3 = C/(3W)
  const float P = (3.f * W - C * C) * (iw * iw) * (1.f / 3.f);  // (3W - C^2)/(3W^2)
  // Q = (-2C^3 + 9CW - 27 s W^2) / (27 W^3)
  const float Q = (fmaf(-2.f * C * C, C, 9.f * C * W) * (iw * iw * iw) - 27.f * s * iw) * (1.f / 27.f);
  const float disc = fmaf(4.f * P * P, P, 27.f * Q * Q);  // 4P^3 + 27Q^2 (< 0: three real roots)
  if (P < 0.f && disc < 0.f) {
    const float m = 2.f * sqrtf(-P * (1.f / 3.f));
    float arg = 3.f * Q / (P * m);                             // (3Q/(2P)) sqrt(-3/P)
    arg = fminf(1.f, fmaxf(-1.f, arg));
    const float th = acosf(arg) * (1.f / 3.f);
    float x3 = fmaf(m, cosf(th), shift);                       // largest
    float x1 = fmaf(m, cosf(th - 2.f * kTwoPi / 3.f), shift);   // smallest
    x3 = newton_cubic(x3, W, C, s);
    if (!(x1 > 0.f)) return x3;
    x1 = newton_cubic(x1, W, C, s);
    // h(x3) - h(x1)
    const float dh = logf(x3 / x1) + s * (1.f / x3 - 1.f / x1) + 0.5f * W * (x3 * x3 - x1 * x1) - C * (x3 - x1);
    return dh < 0.f ? x3 : x1;
  }
  float t;
  if (P > 0.f) {
    const float sq = sqrtf(P * (1.f / 3.f));
    t = -2.f * sq * sinhf(asinhf((3.f * Q / (2.f * P)) / sq) * (1.f / 3.f));
  } else if (P < 0.f) {
    const float sq = sqrtf(-P * (1.f / 3.f));
    const float arg = fmaxf(1.f, (-3.f * fabsf(Q) / (2.f * P)) / sq);
    t = -2.f * copysignf(1.f, Q) * sq * coshf(acoshf(arg) * (1.f / 3.f));
  } else {
    t = -cbrtf(Q);
  }
  float r = t + shift;
  if (!(r > 0.f)) r = s;  // cancellation guard; Newton recovers the root
  return newton_cubic(r, W, C, s);
}

// Same root, solved first by Newton from `r_start` (the pixel's entry value, close to the
// update) when f is monotone (C^2 <= 3W: a single real root, so Newton cannot pick another
// one).  Six steps: starts within a factor 0.7 of the root need five, and a warp pays for
// the closed form if any one of its lanes falls back.  Accepted when the last step changed r
// by less than 2^-20 relative; otherwise, and whenever f is not monotone, the closed form
// above decides.
__device__ __forceinline__ float icd_root_from(float W, float C, float s, float r_start) {
  if (W > 0.f && C * C <= 3.f * W && r_start > 0.f) {
    float r = r_start;
    float step = 0.f;
#pragma unroll
    for (int it = 0; it < 6; ++it) {
      const float f = fmaf(fmaf(fmaf(W, r, -C), r, 1.f), r, -s);
      const float fp = fmaf(fmaf(3.f * W, r, -2.f * C), r, 1.f);  // >= 1 - C^2/(3W) >= 0
      step = f * hw_rcp(fp);
      r -= step;
    }
    if (r > 0.f && fabsf(step) <= 9.5367431640625e-7f * r) return r;
  }
  return icd_root(W, C, s);
}

// ------------------------------------------------------------------- TMA and mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> this CTA's shared memory, completing on `bar`.  Both addresses
// 16-byte aligned, `bytes` a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` polls (each poll may suspend briefly) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Split cluster barrier: every thread arrives (release: its earlier shared-memory writes,
// remote ones included, become visible to the cluster) and later waits (acquire); work between
// the two must not read what other CTAs write before arriving.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Programmatic dependent launch (sm_90+).  `grid_dep_launch` lets the next kernel of the
// stream (launched with programmatic stream serialization) start its independent prologue;
// `grid_dep_wait` blocks until every prerequisite grid has completed and its memory is visible
// (a no-op for a kernel launched without the attribute).
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace ddh
