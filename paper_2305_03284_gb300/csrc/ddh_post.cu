// Post-step kernel of two optional M-step extensions (one CTA per stream, after the frame's
// step kernel on the same stream, programmatic dependent launch).
//
// Phase prior.  The paper names p(phi) in Eq. 2 and leaves its form to earlier work; here the
// tile phases phi_t (phase constant on G x G tiles) carry a Gaussian MRF on the wrapped
// differences of 8-neighbour tiles, with precision lam and the reflectance prior's neighbour
// weights.  With z = F mu and v_t = sum_{i in t} a_i y~_i conj(z_i), the phase part of the EM
// M-step is then
//     f(phi) = -(2/sigma^2) sum_t |v_t| cos(phi_t - angle v_t) + (lam/2) sum_{t~s} b_ts wrap(phi_t - phi_s)^2
// over the tiles that hold a pupil pixel and a non-zero v_t.  Starting from the prior-free
// tile angles (the step kernel's output), each of `sweeps` 4-colour ICD sweeps gives every
// tile the minimiser of a quadratic majoriser of its 1-D function: 1 - cos x is bounded by
// sin(x0)/(2 x0) x^2 + const about x0 = wrap(phi_t - angle v_t), and wrap(d)^2 by
// (d - 2 pi k)^2 with k the current branch; the result is wrapped into (-pi, pi].
//
// Noise variance.  sigma^2 of Eq. 1's noise is re-estimated by its EM M-step,
//     sigma^2 = (1/|P|) sum_{i in P} |y~_i - e^{j phi_i} z_i|^2 + (1/M) sum_j C_jj,
// whose pupil residual is sum_t (E_t - 2 |v_t| cos(phi_t - angle v_t)) with
// E_t = sum_{i in t} a_i (|y~_i|^2 + |z_i|^2) (the step kernel's partial sums at the tile
// angles when there is no prior).  The value goes to aux[0], which the next frame's step
// kernel reads after its dependency wait.
//
// All sums run in a fixed order.  A frame the step kernel dropped (aux[1] == 0) leaves the
// state untouched.
#include <mutex>

#include "ddh_device.cuh"
#include "ddh_kernels.cuh"

namespace ddh {
namespace {

constexpr int kPostThreads = 1024;

__global__ void __launch_bounds__(kPostThreads, 1) k_ddh_post(const __grid_constant__ PostArgs a) {
  grid_dep_launch();
  grid_dep_wait();
  float* aux = a.aux;
  if (aux[1] == 0.f) return;  // the step dropped this frame
  extern __shared__ float sm[];
  __shared__ float red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float nv = aux[0];
  const int n = a.n, gs = a.gs, G = 1 << gs, NT = n >> gs, nt = a.nt, t0 = a.t_lo, nb = nt * nt;
  const float4* tiles = reinterpret_cast<const float4*>(aux + kAuxTiles);
  float res = 0.f;
  if (a.prior) {
    float* kap = sm;            // 2 |v_t| / sigma^2; -1 for a tile outside the prior's graph
    float* th = sm + nb;        // angle v_t
    float* ph = sm + 2 * nb;    // current tile phase
    for (int i = tid; i < nb; i += kPostThreads) {
      const int T = t0 + i / nt, X = t0 + i % nt;
      kap[i] = -1.f;
      th[i] = 0.f;
      ph[i] = 0.f;
      if (!tile_in_pupil(T, X, gs, n, a.ap_lim)) continue;
      const float4 v = tiles[T * NT + X];
      if (v.x == 0.f && v.y == 0.f) continue;
      kap[i] = 2.f * sqrtf(fmaf(v.x, v.x, v.y * v.y)) / nv;
      th[i] = atan2f(v.y, v.x);
      ph[i] = th[i];
    }
    __syncthreads();
    for (int sweep = 0; sweep < a.sweeps; ++sweep) {
      for (int c = 0; c < 4; ++c) {  // colours (x % 2, y % 2) = (0,0), (1,0), (0,1), (1,1)
        const int cx = c & 1, cy = c >> 1;
        for (int i = tid; i < nb; i += kPostThreads) {
          const int ti = i / nt, xi = i - ti * nt;
          if (((t0 + xi) & 1) != cx || ((t0 + ti) & 1) != cy || kap[i] < 0.f) continue;
          const float p0 = ph[i];
          const float x0 = wrap_pi(p0 - th[i]);
          const float c0 = x0 != 0.f ? sinf(x0) / (2.f * x0) : 0.5f;
          float ws = 0.f, ss = 0.f;
#pragma unroll
          for (int nbr = 0; nbr < 8; ++nbr) {
            const int dy = nbr < 2 ? (nbr == 0 ? -1 : 1) : (nbr < 4 ? 0 : (nbr < 6 ? -1 : 1));
            const int dx = nbr < 2 ? 0 : (nbr < 4 ? (nbr == 2 ? -1 : 1) : ((nbr & 1) ? 1 : -1));
            const float b = nbr < 4 ? kBnn : kBdiag;
            const int t2 = ti + dy, x2 = xi + dx;
            if (t2 < 0 || t2 >= nt || x2 < 0 || x2 >= nt) continue;
            const int j = t2 * nt + x2;
            if (kap[j] < 0.f) continue;
            ws += b;
            ss = fmaf(b, p0 - wrap_pi(p0 - ph[j]), ss);
          }
          const float kc = 2.f * kap[i] * c0;
          const float den = fmaf(a.lam, ws, kc);
          if (den > 0.f) ph[i] = wrap_pi(fmaf(kc, p0 - x0, a.lam * ss) / den);
        }
        __syncthreads();
      }
    }
    // the tile phase on the tile's pupil pixels, and the pupil residual at the final phases
    for (int i = tid; i < nb; i += kPostThreads) {
      const int T = t0 + i / nt, X = t0 + i % nt;
      if (!tile_in_pupil(T, X, gs, n, a.ap_lim)) continue;
      const float4 v = tiles[T * NT + X];
      if (kap[i] < 0.f) {
        res += v.z;  // no data in the tile (v_t = 0): its residual is E_t
        continue;
      }
      const float p = ph[i];
      for (int j = 0; j < G; ++j) {
        const int y = (T << gs) + j, dy2 = ap_dist2(y, n);
        for (int m = 0; m < G; ++m) {
          const int x = (X << gs) + m;
          if (ap_dist2(x, n) + dy2 <= a.ap_lim) a.phi[static_cast<size_t>(y) * n + x] = p;
        }
      }
      res += v.z - 2.f * sqrtf(fmaf(v.x, v.x, v.y * v.y)) * cosf(p - th[i]);
    }
  }
  if (a.noise_update) {
    res = warp_sum(res);
    if (lane == 0) red[warp] = res;
    __syncthreads();
    if (tid == 0) {
      float sr = 0.f, sc = 0.f;
      if (a.prior)
        for (int w = 0; w < kPostThreads / 32; ++w) sr += red[w];
      for (int k = 0; k < a.ctas; ++k) {
        if (!a.prior) sr += aux[kAuxPart + 2 * k];
        sc += aux[kAuxPart + 2 * k + 1];
      }
      aux[0] = fmaxf(fmaf(sr, a.inv_ap_count, sc * a.inv_m), a.nv_floor);
    }
  }
}

std::once_flag g_post_once[64];
cudaError_t g_post_attr[64];

}  // namespace

cudaError_t launch_post(const PostArgs& a, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  // the largest tile box (N = 256, G = 2, pupil of diameter N) holds 3 x 128^2 floats
  std::call_once(g_post_once[dev], [dev] {
    g_post_attr[dev] = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_ddh_post),
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 128 * 128 * 4);
  });
  if (g_post_attr[dev] != cudaSuccess) return g_post_attr[dev];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1, 1, 1);
  cfg.blockDim = dim3(kPostThreads, 1, 1);
  cfg.dynamicSmemBytes = a.prior ? static_cast<size_t>(3) * a.nt * a.nt * sizeof(float) : 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_ddh_post, a);
}

}  // namespace ddh
