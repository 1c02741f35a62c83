// Post-step kernel of two optional M-step extensions (one cluster of 8 CTAs per stream, after
// the frame's step kernel on the same stream, programmatic dependent launch; a batch's streams
// share one launch, blockIdx.y = stream).
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
#include <cooperative_groups.h>

#include "ddh_device.cuh"
#include "ddh_kernels.cuh"

namespace cg = cooperative_groups;

namespace ddh {
namespace {

constexpr int kPostCluster = 8;   // CTAs; the tile box's rows are split into 8 contiguous blocks
constexpr int kPostThreads = 256;
constexpr int kPostCols = kPostMaxTiles;  // the prior's tile box is at most 128 x 128 tiles
constexpr int kPostRows = kPostCols / kPostCluster;

__global__ void __cluster_dims__(kPostCluster, 1, 1) __launch_bounds__(kPostThreads)
    k_ddh_post(const __grid_constant__ PostBatch b) {
  const PostArgs& a = b.a[blockIdx.y];
  grid_dep_launch();
  grid_dep_wait();
  float* aux = a.aux;
  if (aux[1] == 0.f) return;  // the step dropped this frame (the same for every CTA)
  cg::cluster_group cluster = cg::this_cluster();
  const int q = static_cast<int>(cluster.block_rank());
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // kap: 2 |v_t| / sigma^2 (-1: tile outside the prior's graph) of this CTA's rows and the row
  // above and below; th: angle v_t and ph: the current phase of this CTA's rows
  __shared__ float kap[(kPostRows + 2) * kPostCols];
  __shared__ float th[kPostRows * kPostCols];
  __shared__ float ph[kPostRows * kPostCols];
  __shared__ float red[kPostThreads / 32];
  __shared__ float part[kPostCluster];  // in CTA 0: every CTA's pupil residual
  const float nv = aux[0];
  const int n = a.n, gs = a.gs, G = 1 << gs, NT = n >> gs, nt = a.nt, t0 = a.t_lo;
  const int rp = (nt + kPostCluster - 1) / kPostCluster;
  const int r0 = min(q * rp, nt), r1 = min(nt, r0 + rp);  // this CTA's box rows [r0, r1)
  const float4* tiles = reinterpret_cast<const float4*>(aux + kAuxTiles);
  float res = 0.f;
  if (a.prior) {
    for (int i = tid; i < (rp + 2) * nt; i += kPostThreads) {
      const int lr = i / nt, xi = i - lr * nt, br = r0 - 1 + lr;
      float kv = -1.f, tv = 0.f;
      if (br >= 0 && br <= r1 && br < nt) {
        const int T = t0 + br, X = t0 + xi;
        if (tile_in_pupil(T, X, gs, n, a.ap_lim)) {
          const float4 v = tiles[T * NT + X];
          if (v.x != 0.f || v.y != 0.f) {
            kv = 2.f * sqrtf(fmaf(v.x, v.x, v.y * v.y)) / nv;
            tv = atan2f(v.y, v.x);
          }
        }
      }
      kap[i] = kv;
      if (br >= r0 && br < r1) {
        th[(br - r0) * nt + xi] = tv;
        ph[(br - r0) * nt + xi] = tv;  // the prior-free tile angle (the step kernel's output)
      }
    }
    cluster.sync();
    for (int sweep = 0; sweep < a.sweeps; ++sweep) {
      for (int c = 0; c < 4; ++c) {  // colours (x % 2, y % 2) = (0,0), (1,0), (0,1), (1,1)
        const int cx = c & 1, cy = c >> 1;
        const int by = (cy - (t0 + r0)) & 1, bx = (cx - t0) & 1;  // first row / column of the colour
        const int nrow = (r1 - r0 - by + 1) / 2, ncol = (nt - bx + 1) / 2;
        for (int k = tid; k < nrow * ncol; k += kPostThreads) {
          const int br = r0 + by + 2 * (k / ncol), xi = bx + 2 * (k % ncol);
          const float kv = kap[(br - r0 + 1) * nt + xi];
          if (kv < 0.f) continue;
          const int li = (br - r0) * nt + xi;
          const float p0 = ph[li];
          const float x0 = wrap_pi(p0 - th[li]);
          const float c0 = x0 != 0.f ? sinf(x0) / (2.f * x0) : 0.5f;
          float ws = 0.f, ss = 0.f;
#pragma unroll
          for (int nbr = 0; nbr < 8; ++nbr) {  // N, S, W, E, NW, NE, SW, SE
            const int dy = nbr < 2 ? (nbr == 0 ? -1 : 1) : (nbr < 4 ? 0 : (nbr < 6 ? -1 : 1));
            const int dx = nbr < 2 ? 0 : (nbr < 4 ? (nbr == 2 ? -1 : 1) : ((nbr & 1) ? 1 : -1));
            const float b = nbr < 4 ? kBnn : kBdiag;
            const int t2 = br + dy, x2 = xi + dx;
            if (t2 < 0 || t2 >= nt || x2 < 0 || x2 >= nt) continue;
            if (kap[(t2 - r0 + 1) * nt + x2] < 0.f) continue;
            float pj;
            if (t2 >= r0 && t2 < r1) {
              pj = ph[(t2 - r0) * nt + x2];
            } else {  // a neighbouring CTA's row (it does not change during this colour)
              const int owner = t2 / rp;
              pj = cluster.map_shared_rank(ph, owner)[(t2 - owner * rp) * nt + x2];
            }
            ws += b;
            ss = fmaf(b, p0 - wrap_pi(p0 - pj), ss);
          }
          const float kc = 2.f * kv * c0;
          const float den = fmaf(a.lam, ws, kc);
          if (den > 0.f) ph[li] = wrap_pi(fmaf(kc, p0 - x0, a.lam * ss) / den);
        }
        cluster.sync();  // this colour's phases are visible to the neighbouring rows' owners
      }
    }
    // the tile phase on its pupil pixels, and the pupil residual at the final phases
    for (int i = tid; i < (r1 - r0) * nt; i += kPostThreads) {
      const int lr = i / nt, xi = i - lr * nt;
      const int T = t0 + r0 + lr, X = t0 + xi;
      if (!tile_in_pupil(T, X, gs, n, a.ap_lim)) continue;
      const float4 v = tiles[T * NT + X];
      if (kap[(lr + 1) * nt + xi] < 0.f) {
        res += v.z;  // no data in the tile (v_t = 0): its residual is E_t
        continue;
      }
      const float p = ph[lr * nt + xi];
      for (int j = 0; j < G; ++j) {
        const int y = (T << gs) + j, dy2 = ap_dist2(y, n);
        for (int m = 0; m < G; ++m) {
          const int x = (X << gs) + m;
          if (ap_dist2(x, n) + dy2 <= a.ap_lim) a.phi[static_cast<size_t>(y) * n + x] = p;
        }
      }
      res += v.z - 2.f * sqrtf(fmaf(v.x, v.x, v.y * v.y)) * cosf(p - th[lr * nt + xi]);
    }
    if (a.noise_update) {  // this CTA's residual into CTA 0, in CTA order
      res = warp_sum(res);
      if (lane == 0) red[warp] = res;
      __syncthreads();
      if (tid == 0) {
        float sr = 0.f;
        for (int w = 0; w < kPostThreads / 32; ++w) sr += red[w];
        cluster.map_shared_rank(part, 0)[q] = sr;
      }
      cluster.sync();
    }
  }
  if (a.noise_update && q == 0) {
    // the step kernel's partial sums are fetched in parallel, then added in CTA order
    __shared__ float pa[2 * kAuxParts];
    if (tid < 2 * a.ctas) pa[tid] = aux[kAuxPart + tid];
    __syncthreads();
    if (tid == 0) {
      float sr = 0.f, sc = 0.f;
      if (a.prior)
        for (int k = 0; k < kPostCluster; ++k) sr += part[k];
      for (int k = 0; k < a.ctas; ++k) {
        if (!a.prior) sr += pa[2 * k];
        sc += pa[2 * k + 1];
      }
      aux[0] = fmaxf(fmaf(sr, a.inv_ap_count, sc * a.inv_m), a.nv_floor);
    }
  }
}

}  // namespace

cudaError_t launch_post_batch(const PostBatch& b, cudaStream_t st) {
  if (b.count < 1 || b.count > kMaxBatch) return cudaErrorInvalidValue;
  for (int i = 0; i < b.count; ++i)
    if ((b.a[i].prior && b.a[i].nt > kPostCols) || b.a[i].ctas > kAuxParts) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kPostCluster, b.count, 1);
  cfg.blockDim = dim3(kPostThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_ddh_post, b);
}

cudaError_t launch_post(const PostArgs& a, cudaStream_t st) {
  PostBatch b{};
  b.a[0] = a;
  b.count = 1;
  return launch_post_batch(b, st);
}

}  // namespace ddh
