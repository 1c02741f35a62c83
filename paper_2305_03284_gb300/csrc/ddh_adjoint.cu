// Hand-written adjoint of one DDH-MBIR frame step (one EM iteration, per-pixel phase).
//
// Given dL/dr_n and dL/dphi_n for the frame's outputs, the kernels below produce dL/dr_{n-1},
// dL/dphi_{n-1} and the frame's contribution to dL/dsigma_r, dL/dp (q-GGMRF scale and shape)
// and dL/dsigma^2, by the chain rule through the stages of the step in reverse:
//   phase M-step phi = angle(v), v = y~ conj(z), z = F mu      (v_bar = phi_bar i v / |v|^2)
//   ICD sweep, colours 3..0: r_i = root(W_i, C_i, s_i) differentiated implicitly,
//       W = sum beta, C = sum beta r_j, beta_ij = b_ij w(r0_i - r0_j; sigma_r, p)
//   E-step w = r0/(r0 + s2), mu = w b, s = |mu|^2 + s2 w; r-init (Eq. 3) with its floor
//   back-projection b = F^H(a e^{-j phi'} y~), RemoveTipTilt phi' = phi - plane
// The forward intermediates come from ddh_step_trace of the same frame from the same state
// (the caller's per-frame checkpoint).  Complex gradients are dL/dRe + i dL/dIm.  All sums are
// in a fixed order (deterministic).  The caller provides every buffer, workspace included.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "../../include/ddh.h"
#include "ddh_device.cuh"
#include "ddh_internal.h"
#include "ddh_kernels.cuh"

namespace ddh {
namespace {

constexpr int kBwThreads = 256;
constexpr int kBwMaxBlocks = 128;  // the partial-sum area holds 2 + 3 floats per block
constexpr int kBwRedFloats = 1024;

struct BwParams {
  int n, ap_lim, tilt_mode;
  float lam1, lam_alpha, noise_var, r_floor;
  float w0, inv_tsig, q_minus_p, q_over_p, q, p, sigma, log_t;
  float gx_scale, gy_scale;  // 1/|P_x|, 1/|P_y| (0 when there is no pair)
};

struct BwBuffers {
  const float2* y;
  const float* r_prev;
  const float* phi_prev;
  const float* trace;
  const float* r_new;
  const float* r_bar;
  const float* phi_bar;
  float* r_prev_bar;
  float* phi_prev_bar;
  float* grads;
  // workspace
  float2* cbuf1;  // z_bar -> mu_bar
  float2* cbuf2;  // b_bar -> u_bar
  float* abar;
  float* r0bar;
  float* sbar;
  float* cbar;
  float* wbar;
  float* pg;      // 3 x M per-pixel parameter partials (sigma_r, p, sigma^2)
  float* red;     // block partials: tilt sums (2 per block), then parameter partials (3 per block)
  float4* pairs;  // 4 x M: (w, dw/dD, dw/dsigma_r, dw/dp) of the pair (p, p + dir), D = r0_p - r0_q
};

struct WD {
  float w, dd, ds, dp;
};

// w(D) = rho'(D)/D (q = 2) with its partial derivatives in D, sigma_r and p.
__device__ __forceinline__ WD weight_derivs(float delta, const BwParams& P) {
  const float ad = fabsf(delta);
  const float t = ad * P.inv_tsig;
  const float lt = t > 0.f ? logf(t) : 0.f;
  const float u = t > 0.f ? expf(P.q_minus_p * lt) : 0.f;
  const float A = P.q_over_p + u, B = 1.f + u;
  WD r;
  r.w = P.w0 * A / (B * B);
  const float k = 1.f / A - 2.f / B;
  const float du_dd = ad > 0.f ? P.q_minus_p * u / delta : 0.f;
  r.dd = r.w * k * du_dd;
  const float du_ds = -P.q_minus_p * u / P.sigma;
  r.ds = r.w * (-2.f / P.sigma + k * du_ds);
  const float du_dp = -u * lt;
  r.dp = r.w * (P.log_t + (-P.q / (P.p * P.p) + du_dp) / A - 2.f * du_dp / B);
  return r;
}

__device__ __forceinline__ int colour_of(int row, int col) { return (col & 1) + 2 * (row & 1); }

__device__ __forceinline__ void neighbour(int nb, int& dy, int& dx, float& bij) {
  // order: N, S, W, E, NW, NE, SW, SE (orthogonal weight first four)
  const int dys[8] = {-1, 1, 0, 0, -1, -1, 1, 1};
  const int dxs[8] = {0, 0, -1, 1, -1, 1, -1, 1};
  dy = dys[nb];
  dx = dxs[nb];
  bij = nb < 4 ? kBnn : kBdiag;
}

// Each neighbour pair is stored once, at the pixel p from which the other pixel q lies in one of
// the four "forward" directions S, E, SW, SE (table planes 0..3), with D = r0_p - r0_q.  w, dw/ds
// and dw/dp depend on |D| only and dw/dD is odd in D, so the entry seen from q is the stored one
// with dw/dD negated (bit for bit).  Offsets nb and its opposite share a plane.
__device__ __forceinline__ int pair_plane(int nb) {
  const int planes[8] = {0, 0, 1, 1, 3, 2, 2, 3};
  return planes[nb];
}
__device__ __forceinline__ bool pair_forward(int nb) { return nb == 1 || nb == 3 || nb >= 6; }

// The pair between pixel `a` and its neighbour b = a + offset nb, as seen from `a`.
__device__ __forceinline__ float4 pair_from(const float4* pairs, int M, int nb, int a, int b) {
  if (pair_forward(nb)) return pairs[pair_plane(nb) * M + a];
  float4 e = pairs[pair_plane(nb) * M + b];
  e.y = -e.y;
  return e;
}

// The pair table of the frame: one thread per (plane, pixel).
__global__ void k_bw_pairs(BwParams P, BwBuffers B) {
  grid_dep_launch();
  grid_dep_wait();
  const int n = P.n, M = n * n;
  const float* r0 = B.trace + static_cast<size_t>(6) * M;
  const int fwd[4] = {1, 3, 6, 7};  // S, E, SW, SE
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 4 * M; t += gridDim.x * blockDim.x) {
    const int plane = t / M, i = t - plane * M;
    const int row = i / n, col = i - row * n;
    int dy, dx;
    float bij;
    neighbour(fwd[plane], dy, dx, bij);
    const int rr = row + dy, cc = col + dx;
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rr < n && cc >= 0 && cc < n) {
      const WD wd = weight_derivs(r0[i] - r0[rr * n + cc], P);
      e = make_float4(wd.w, wd.dd, wd.ds, wd.dp);
    }
    B.pairs[t] = e;
  }
}

// phase M-step adjoint; also initialises the accumulators
__global__ void k_bw_phase(BwParams P, BwBuffers B) {
  grid_dep_launch();
  grid_dep_wait();
  const int n = P.n, M = n * n;
  const float* stats = B.trace + static_cast<size_t>(8) * M;
  const float2 mean = make_float2(stats[0], stats[1]);
  const float scale = stats[2];
  const float2* z = reinterpret_cast<const float2*>(B.trace) + 2 * M;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int row = i / n, col = i - row * n;
    float2 zb = make_float2(0.f, 0.f);
    if (ap_dist2(row, n) + ap_dist2(col, n) <= P.ap_lim) {
      const float2 yt = c_scale(c_sub(B.y[i], mean), scale);
      const float2 zz = z[i];
      const float2 v = make_float2(fmaf(yt.x, zz.x, yt.y * zz.y), fmaf(yt.y, zz.x, -yt.x * zz.y));
      const float m2 = c_abs2(v);
      if (m2 > 0.f) {
        const float g = B.phi_bar[i] / m2;
        const float2 vb = make_float2(-v.y * g, v.x * g);  // phi_bar i v / |v|^2
        zb = c_mul(yt, make_float2(vb.x, -vb.y));          // y~ conj(v_bar)
      }
    }
    B.cbuf1[i] = zb;
    B.abar[i] = B.r_bar[i];
    B.r0bar[i] = 0.f;
    B.sbar[i] = 0.f;
    B.pg[i] = 0.f;
    B.pg[M + i] = 0.f;
    B.pg[2 * M + i] = 0.f;
  }
}

// ICD adjoint, pass A for the pixels of colour c: implicit derivative of the root.
__global__ void k_bw_icd_a(BwParams P, BwBuffers B, int c) {
  grid_dep_launch();
  grid_dep_wait();
  const int n = P.n, M = n * n, h = n / 2;
  const float* r0 = B.trace + static_cast<size_t>(6) * M;
  // the colour-c pixels: rows of parity c / 2, columns of parity c % 2
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M / 4; k += gridDim.x * blockDim.x) {
    const int kr = k / h;
    const int row = 2 * kr + (c >> 1), col = 2 * (k - kr * h) + (c & 1);
    const int i = row * n + col;
    const float rn = B.r_new[i];
    float Wsum = 0.f, Csum = 0.f;
    float beta[8], cur[8];
    float4 wd[8];
    bool in[8];
    for (int nb = 0; nb < 8; ++nb) {
      int dy, dx;
      float bij;
      neighbour(nb, dy, dx, bij);
      const int rr = row + dy, cc = col + dx;
      in[nb] = rr >= 0 && rr < n && cc >= 0 && cc < n;
      if (!in[nb]) continue;
      const int j = rr * n + cc;
      wd[nb] = pair_from(B.pairs, M, nb, i, j);
      beta[nb] = bij * wd[nb].x;
      cur[nb] = colour_of(rr, cc) < c ? B.r_new[j] : r0[j];
      Wsum += beta[nb];
      Csum = fmaf(beta[nb], cur[nb], Csum);
    }
    const bool clamped = !(rn > P.r_floor);
    const float gbar = clamped ? 0.f : B.abar[i];
    B.abar[i] = 0.f;
    const float gp = fmaf(fmaf(3.f * Wsum, rn, -2.f * Csum), rn, 1.f);
    const float inv = gbar != 0.f ? gbar / gp : 0.f;
    const float wbar = -inv * rn * rn * rn;
    const float cbar = inv * rn * rn;
    B.sbar[i] = inv;
    B.cbar[i] = cbar;
    B.wbar[i] = wbar;
    float r0b = 0.f, gs = 0.f, gpp = 0.f;
    for (int nb = 0; nb < 8; ++nb) {
      if (!in[nb]) continue;
      int dy, dx;
      float bij;
      neighbour(nb, dy, dx, bij);
      const float bb = fmaf(cbar, cur[nb], wbar) * bij;
      r0b = fmaf(bb, wd[nb].y, r0b);
      gs = fmaf(bb, wd[nb].z, gs);
      gpp = fmaf(bb, wd[nb].w, gpp);
    }
    B.r0bar[i] += r0b;
    B.pg[i] += gs;
    B.pg[M + i] += gpp;
  }
}

// ICD adjoint, pass B: every pixel gathers from its colour-c neighbours.
__global__ void k_bw_icd_b(BwParams P, BwBuffers B, int c) {
  grid_dep_launch();
  grid_dep_wait();
  const int n = P.n, M = n * n;
  const float* r0 = B.trace + static_cast<size_t>(6) * M;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    const int row = j / n, col = j - row * n;
    const int cj = colour_of(row, col);
    if (cj == c) continue;
    const float cur = cj < c ? B.r_new[j] : r0[j];
    float ab = 0.f, r0b = 0.f;
    for (int nb = 0; nb < 8; ++nb) {
      int dy, dx;
      float bij;
      neighbour(nb, dy, dx, bij);
      const int rr = row + dy, cc = col + dx;
      if (rr < 0 || rr >= n || cc < 0 || cc >= n || colour_of(rr, cc) != c) continue;
      const int i = rr * n + cc;
      // the pair as pixel i saw it (D = r0_i - r0_j): stored at j when i lies forward of j
      float4 wd;
      if (pair_forward(nb)) {
        wd = B.pairs[pair_plane(nb) * M + j];
        wd.y = -wd.y;
      } else {
        wd = B.pairs[pair_plane(nb) * M + i];
      }
      const float ci = B.cbar[i];
      ab = fmaf(ci, bij * wd.x, ab);
      r0b = fmaf(fmaf(ci, cur, B.wbar[i]) * bij, wd.y, r0b);
    }
    B.abar[j] += ab;
    B.r0bar[j] -= r0b;
  }
}

// E-step and r-init adjoint.
__global__ void k_bw_estep(BwParams P, BwBuffers B) {
  grid_dep_launch();
  grid_dep_wait();
  const int n = P.n, M = n * n;
  const float2* bt = reinterpret_cast<const float2*>(B.trace);
  const float2* mut = bt + M;
  const float* r0 = B.trace + static_cast<size_t>(6) * M;
  const float s2 = P.noise_var;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const float2 b = bt[i], mu = mut[i];
    const float r = r0[i];
    const float sb = B.sbar[i];
    float r0b = B.r0bar[i] + B.abar[i];
    const float2 mub = make_float2(fmaf(2.f * sb, mu.x, B.cbuf1[i].x), fmaf(2.f * sb, mu.y, B.cbuf1[i].y));
    const float d = r + s2;
    const float w = r / d;
    const float wb = fmaf(mub.x, b.x, mub.y * b.y) + sb * s2;
    float2 bb = c_scale(mub, w);
    B.pg[2 * M + i] = fmaf(sb, w, wb * (-r / (d * d)));
    r0b = fmaf(wb, s2 / (d * d), r0b);
    const float pre = fmaf(P.lam1, B.r_prev[i], P.lam_alpha * c_abs2(b));
    const bool live = pre > P.r_floor;
    B.r_prev_bar[i] = live ? P.lam1 * r0b : 0.f;
    if (live) {
      const float g = 2.f * P.lam_alpha * r0b;
      bb = make_float2(fmaf(g, b.x, bb.x), fmaf(g, b.y, bb.y));
    }
    B.cbuf2[i] = bb;
  }
}

// Back-projection adjoint: phi'_bar = Im(conj(u_bar) u) on the pupil, plus block partials of
// the tilt adjoints t_x_bar = -sum phi'_bar (x - c), t_y_bar = -sum phi'_bar (y - c).
__global__ void k_bw_tilt_a(BwParams P, BwBuffers B) {
  grid_dep_launch();
  grid_dep_wait();
  const int n = P.n, M = n * n;
  const float* stats = B.trace + static_cast<size_t>(8) * M;
  const float2 mean = make_float2(stats[0], stats[1]);
  const float scale = stats[2], tx = stats[3], ty = stats[4];
  const float cc = 0.5f * static_cast<float>(n - 1);
  float sx = 0.f, sy = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int row = i / n, col = i - row * n;
    float pb = 0.f;
    if (ap_dist2(row, n) + ap_dist2(col, n) <= P.ap_lim) {
      float ph = B.phi_prev[i];
      if (P.tilt_mode) ph = wrap_pi(ph - fmaf(tx, static_cast<float>(col) - cc, ty * (static_cast<float>(row) - cc)));
      const float2 yt = c_scale(c_sub(B.y[i], mean), scale);
      float sn, cs;
      sincosf(ph, &sn, &cs);
      const float2 u = make_float2(fmaf(yt.x, cs, yt.y * sn), fmaf(yt.y, cs, -yt.x * sn));
      const float2 ub = B.cbuf2[i];
      pb = ub.x * u.y - ub.y * u.x;  // Im(conj(u_bar) u)
      sx = fmaf(-pb, static_cast<float>(col) - cc, sx);
      sy = fmaf(-pb, static_cast<float>(row) - cc, sy);
    }
    B.phi_prev_bar[i] = pb;
  }
  __shared__ float shx[kBwThreads], shy[kBwThreads];
  shx[threadIdx.x] = sx;
  shy[threadIdx.x] = sy;
  __syncthreads();
  for (int o = kBwThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      shx[threadIdx.x] += shx[threadIdx.x + o];
      shy[threadIdx.x] += shy[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    B.red[2 * blockIdx.x] = shx[0];
    B.red[2 * blockIdx.x + 1] = shy[0];
  }
}

// Tilt-estimate adjoint: phi_bar(x+1) += t_bar/|P|, phi_bar(x) -= t_bar/|P| for every
// aperture pair (every block sums the tilt partials in the same order), and each block's
// partial sums of the three per-pixel parameter partials (fixed order within the block).
__global__ void k_bw_tilt_b(BwParams P, BwBuffers B, int blocks) {
  grid_dep_launch();
  grid_dep_wait();
  const int n = P.n, M = n * n;
  __shared__ float g[2];
  __shared__ float sh[3][kBwThreads];
  __shared__ float tp[2 * kBwMaxBlocks];
  // the tilt partials are fetched in parallel, then summed in block order by one thread
  for (int i = threadIdx.x; i < 2 * blocks; i += blockDim.x) tp[i] = B.red[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    float tx = 0.f, ty = 0.f;
    for (int b = 0; b < blocks; ++b) {
      tx += tp[2 * b];
      ty += tp[2 * b + 1];
    }
    g[0] = P.tilt_mode ? tx * P.gx_scale : 0.f;
    g[1] = P.tilt_mode ? ty * P.gy_scale : 0.f;
  }
  __syncthreads();
  const float gx = g[0], gy = g[1];
  float acc[3] = {0.f, 0.f, 0.f};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] += B.pg[k * M + i];
    const int row = i / n, col = i - row * n;
    const int dy2 = ap_dist2(row, n);
    if (dy2 + ap_dist2(col, n) > P.ap_lim) {
      B.phi_prev_bar[i] = 0.f;
      continue;
    }
    float add = 0.f;
    if (col > 0 && dy2 + ap_dist2(col - 1, n) <= P.ap_lim) add += gx;      // pair (x-1, x): right end
    if (col + 1 < n && dy2 + ap_dist2(col + 1, n) <= P.ap_lim) add -= gx;  // pair (x, x+1): left end
    const int dx2 = ap_dist2(col, n);
    if (row > 0 && ap_dist2(row - 1, n) + dx2 <= P.ap_lim) add += gy;
    if (row + 1 < n && ap_dist2(row + 1, n) + dx2 <= P.ap_lim) add -= gy;
    B.phi_prev_bar[i] += add;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = kBwThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) B.red[2 * kBwMaxBlocks + 3 * blockIdx.x + k] = sh[k][0];
}

// The parameter gradients: the blocks' partials summed in block order.
__global__ void k_bw_grads(BwBuffers B, int blocks) {
  grid_dep_launch();
  grid_dep_wait();
  __shared__ float pp[3 * kBwMaxBlocks];
  // the partials are fetched in parallel, then each sum runs in block order
  for (int i = threadIdx.x; i < 3 * blocks; i += blockDim.x) pp[i] = B.red[2 * kBwMaxBlocks + i];
  __syncthreads();
  if (threadIdx.x < 3) {
    float acc = 0.f;
    for (int b = 0; b < blocks; ++b) acc += pp[3 * b + threadIdx.x];
    B.grads[threadIdx.x] += acc;
  }
}

// Launch with programmatic stream serialization (each kernel waits for its predecessor itself).
template <typename... Params, typename... Args>
cudaError_t launch_bw(void (*kern)(Params...), int blocks, int threads, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(blocks), 1, 1);
  cfg.blockDim = dim3(static_cast<unsigned>(threads), 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace
}  // namespace ddh

extern "C" {

size_t ddh_backward_workspace_bytes(int n) {
  if (n != 32 && n != 64 && n != 128 && n != 256) return 0;
  const size_t M = static_cast<size_t>(n) * n;
  return sizeof(float) * (4 * M + 5 * M + 3 * M + ddh::kBwRedFloats + 16 * M);
}

}  // extern "C"

int ddh_internal_step_backward(int n, const ddh_params* prm, const void* twiddle, void* stream_v, const void* y,
                               const float* r_prev, const float* phi_prev, const float* trace, const float* r_new,
                               const float* r_bar, const float* phi_bar, float* r_prev_bar, float* phi_prev_bar,
                               float* grads, void* workspace) {
  using namespace ddh;
  cudaStream_t st = static_cast<cudaStream_t>(stream_v);
  const size_t M = static_cast<size_t>(n) * n;
  BwParams P{};
  P.n = n;
  const double d = prm->aperture_diam;
  P.ap_lim = static_cast<int>(std::floor(d * d));
  P.tilt_mode = prm->tilt_mode;
  P.lam1 = static_cast<float>(1.0 - static_cast<double>(prm->lambda));
  P.lam_alpha = static_cast<float>(static_cast<double>(prm->lambda) * prm->alpha);
  P.noise_var = prm->noise_var;
  P.r_floor = prm->r_floor;
  const double ts = static_cast<double>(prm->prior_T) * prm->prior_sigma;
  P.w0 = static_cast<float>(std::pow(ts, static_cast<double>(prm->prior_p) - 2.0) *
                            std::pow(static_cast<double>(prm->prior_sigma), -static_cast<double>(prm->prior_p)));
  P.inv_tsig = static_cast<float>(1.0 / ts);
  P.q_minus_p = static_cast<float>(static_cast<double>(prm->prior_q) - prm->prior_p);
  P.q_over_p = static_cast<float>(static_cast<double>(prm->prior_q) / prm->prior_p);
  P.q = prm->prior_q;
  P.p = prm->prior_p;
  P.sigma = prm->prior_sigma;
  P.log_t = static_cast<float>(std::log(static_cast<double>(prm->prior_T)));
  // aperture pair counts of the tip/tilt regression (integer geometry)
  int64_t px = 0, py = 0;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      const int64_t dy = 2 * r - (n - 1), dx = 2 * c - (n - 1);
      if (dx * dx + dy * dy > P.ap_lim) continue;
      const int64_t dxn = 2 * (c + 1) - (n - 1), dyn = 2 * (r + 1) - (n - 1);
      if (c + 1 < n && dxn * dxn + dy * dy <= P.ap_lim) ++px;
      if (r + 1 < n && dx * dx + dyn * dyn <= P.ap_lim) ++py;
    }
  P.gx_scale = px > 0 ? static_cast<float>(1.0 / static_cast<double>(px)) : 0.f;
  P.gy_scale = py > 0 ? static_cast<float>(1.0 / static_cast<double>(py)) : 0.f;

  BwBuffers B{};
  B.y = static_cast<const float2*>(y);
  B.r_prev = r_prev;
  B.phi_prev = phi_prev;
  B.trace = trace;
  B.r_new = r_new;
  B.r_bar = r_bar;
  B.phi_bar = phi_bar;
  B.r_prev_bar = r_prev_bar;
  B.phi_prev_bar = phi_prev_bar;
  B.grads = grads;
  float* ws = static_cast<float*>(workspace);
  B.cbuf1 = reinterpret_cast<float2*>(ws);
  B.cbuf2 = reinterpret_cast<float2*>(ws + 2 * M);
  B.abar = ws + 4 * M;
  B.r0bar = ws + 5 * M;
  B.sbar = ws + 6 * M;
  B.cbar = ws + 7 * M;
  B.wbar = ws + 8 * M;
  B.pg = ws + 9 * M;
  B.red = ws + 12 * M;
  B.pairs = reinterpret_cast<float4*>(ws + 12 * M + kBwRedFloats);  // 16-byte aligned
  // grid-stride kernels over the N x N image: as many blocks as pixels fill, up to 128
  const int blocks = static_cast<int>(std::min<size_t>(kBwMaxBlocks, (M + kBwThreads - 1) / kBwThreads));
  cudaError_t e = launch_bw(k_bw_phase, blocks, kBwThreads, st, P, B);
  if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
  Fft2Args f{};
  f.in = B.cbuf1;
  f.out = B.cbuf1;
  f.tw = static_cast<const float2*>(twiddle);
  f.inverse = 1;
  e = launch_fft2(n, f, st);  // mu_bar = F^H z_bar
  if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
  const int pair_blocks = static_cast<int>((4 * M + kBwThreads - 1) / kBwThreads);
  const int colour_blocks = static_cast<int>((M / 4 + kBwThreads - 1) / kBwThreads);
  const int pixel_blocks = static_cast<int>((M + kBwThreads - 1) / kBwThreads);
  if (e == cudaSuccess) e = launch_bw(k_bw_pairs, pair_blocks, kBwThreads, st, P, B);
  for (int c = 3; c >= 0 && e == cudaSuccess; --c) {
    e = launch_bw(k_bw_icd_a, colour_blocks, kBwThreads, st, P, B, c);
    if (e == cudaSuccess) e = launch_bw(k_bw_icd_b, pixel_blocks, kBwThreads, st, P, B, c);
  }
  if (e == cudaSuccess) e = launch_bw(k_bw_estep, blocks, kBwThreads, st, P, B);
  if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
  f.in = B.cbuf2;
  f.out = B.cbuf2;
  f.inverse = 0;
  e = launch_fft2(n, f, st);  // u_bar = F b_bar
  if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
  e = launch_bw(k_bw_tilt_a, blocks, kBwThreads, st, P, B);
  if (e == cudaSuccess) e = launch_bw(k_bw_tilt_b, blocks, kBwThreads, st, P, B, blocks);
  if (e == cudaSuccess) e = launch_bw(k_bw_grads, 1, 128, st, B, blocks);
  if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
  e = cudaGetLastError();
  if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
  return DDH_OK;
}

// ---- allocation-free variant -----------------------------------------------------------------
// Scratch for ddh_step_backward_noalloc: a file-scope device array, present on every device
// that loads the library until the process exits.  It holds the backward workspace of grids up
// to 128 x 128 (28 N^2 + 1024 floats = 1796 KiB).  Host code must not pass the array's name to a
// kernel (on the host it is only a stand-in); its device address is looked up with the device
// current, once per device and CUDA context: a context created after a device reset (a new
// context ID) gets a fresh lookup, so a stale address is never passed to the kernels.
namespace {
constexpr int kNoAllocMaxN = 128;
constexpr int kNoAllocDevices = 64;
constexpr size_t kNoAllocScratchFloats = 28 * static_cast<size_t>(kNoAllocMaxN) * kNoAllocMaxN + ddh::kBwRedFloats;
static __device__ __align__(256) float g_backward_scratch[kNoAllocScratchFloats];
std::mutex g_scratch_mu;
void* g_scratch_addr[kNoAllocDevices] = {};
unsigned long long g_scratch_ctx[kNoAllocDevices] = {};

// The unique ID of the calling thread's current CUDA context (driver cuCtxGetCurrent and
// cuCtxGetId, reached through the runtime's driver entry points), or 0 if unavailable.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current == nullptr || get_id == nullptr || get_current(&ctx) != 0 || ctx == nullptr) return 0;
  return get_id(ctx, &id) == 0 ? id : 0;
}
}  // namespace

extern "C" int ddh_step_backward_noalloc(ddh_state* s, const void* y, const float* r_prev, const float* phi_prev,
                                         const float* trace, const float* r_new, const float* r_bar,
                                         const float* phi_bar, float* r_prev_bar, float* phi_prev_bar,
                                         float* grads) {
  DdhNvtxRange nv("ddh_step_backward_noalloc");
  const ddh_params* prm = nullptr;
  const void* tw = nullptr;
  void* stream = nullptr;
  int dev = 0;
  if (ddh_internal_state_info(s, &prm, &tw, &stream, &dev) != DDH_OK) return DDH_EINVAL;
  if (r_prev == nullptr || phi_prev == nullptr || r_new == nullptr || r_bar == nullptr || phi_bar == nullptr ||
      r_prev_bar == nullptr || phi_prev_bar == nullptr || grads == nullptr) {
    ddh_internal_set_error("ddh_step_backward_noalloc: null buffer argument");
    return DDH_EINVAL;
  }
  int rc = ddh_internal_backward_check(s, y, trace);
  if (rc != DDH_OK) return rc;
  if (prm->n > kNoAllocMaxN) {
    ddh_internal_set_error("ddh_step_backward_noalloc: grid larger than 128 x 128 (its static scratch is 1796 KiB); "
                           "use ddh_step_backward with a caller workspace");
    return DDH_EINVAL;
  }
  if (dev < 0 || dev >= kNoAllocDevices) {
    ddh_internal_set_error("ddh_step_backward_noalloc: device ordinal beyond the supported 64");
    return DDH_EINVAL;
  }
  DdhDeviceGuard guard(dev);
  cudaError_t e = guard.error();
  if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long ctx = current_context_id();
    if (g_scratch_addr[dev] == nullptr || ctx == 0 || ctx != g_scratch_ctx[dev]) {
      // first call on this device (or in a new context), with the device current
      void* addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_backward_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return ddh_internal_cuda_fail(e);
      }
      g_scratch_addr[dev] = addr;
      g_scratch_ctx[dev] = ctx;
    }
    scratch = g_scratch_addr[dev];
  }
  return ddh_internal_step_backward(prm->n, prm, tw, stream, y, r_prev, phi_prev, trace, r_new, r_bar, phi_bar,
                                    r_prev_bar, phi_prev_bar, grads, scratch);
}
