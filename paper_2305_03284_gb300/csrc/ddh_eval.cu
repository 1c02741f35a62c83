// Strehl ratio (Sec. 5.B) of a stream on the L2-staged path, for the evaluation call
// ddh_strehl: two launches over the stream's scratch image.
#include "ddh_device.cuh"
#include "ddh_eval.cuh"

namespace ddh {

namespace {
constexpr int kEvTr = 8;  // rows per block of the row pass (one warp per row)
constexpr int kEvTc = 8;  // columns per block of the column pass (one warp per column)
constexpr int kEvRowThreads = 32 * kEvTr;
constexpr int kEvColThreads = 32 * kEvTc;
}  // namespace

// ---- Strehl ratio (Sec. 5.B) of a staged stream ---------------------------------------------
// max |F^H(a e^{j(phi_true - phi_est)})|^2 / max |F^H a|^2 with unscaled transforms: the row
// pass forms the pupil field and transforms its rows (one warp per row, kEvTr rows per block;
// rows off the pupil are zero and are neither transformed nor stored), the column pass
// transforms the columns (one warp per column, kEvTc per block, gathered as row segments of kEvTc
// values) and folds the largest |.|^2 into `max_bits`; the caller divides by (sum a)^2.
template <int N>
__global__ void __launch_bounds__(kEvRowThreads) k_l2_strehl_rows(const __grid_constant__ StrehlL2Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* rows = tw + N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  __syncthreads();
  const int rho = blockIdx.x * kEvTr + warp;
  const int dy2 = ap_dist2(rho, N);
  if (dy2 > a.ap_lim) return;
  float2* rb = rows + warp * (N + 4);
  for (int x = lane; x < N; x += 32) {
    float2 v = make_float2(0.f, 0.f);
    if (ap_dist2(x, N) + dy2 <= a.ap_lim) {
      const size_t gi = static_cast<size_t>(rho) * N + x;
      float sn, cs;
      sincosf(a.phi_true[gi] - a.phi_est[gi], &sn, &cs);
      v = make_float2(cs, sn);
    }
    rb[swz(x)] = v;
  }
  __syncwarp();
  fft_row<N, +1>(rb, tw, lane);
  for (int x = lane; x < N; x += 32) a.work[static_cast<size_t>(rho) * N + x] = rb[swz(x)];
}

template <int N>
__global__ void __launch_bounds__(kEvColThreads) k_l2_strehl_cols(const __grid_constant__ StrehlL2Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* cols = tw + N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x0 = blockIdx.x * kEvTc;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  for (int i = threadIdx.x; i < N * kEvTc; i += blockDim.x) {
    const int rho = i / kEvTc, c = i - rho * kEvTc;
    cols[c * (N + 4) + swz(rho)] = ap_dist2(rho, N) <= a.ap_lim ? a.work[static_cast<size_t>(rho) * N + x0 + c]
                                                              : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* cb = cols + warp * (N + 4);
  fft_row<N, +1>(cb, tw, lane);
  float m = 0.f;
  for (int rho = lane; rho < N; rho += 32) m = fmaxf(m, c_abs2(cb[swz(rho)]));
  m = warp_max(m);
  if (lane == 0) atomicMax(a.max_bits, __float_as_uint(m));  // non-negative floats order as their bits
}

cudaError_t launch_strehl_l2(int n, const StrehlL2Args& a, cudaStream_t st) {
  if (n != 512) return cudaErrorInvalidValue;
  constexpr int N = 512;
  const size_t smem_r = sizeof(float2) * (N + kEvTr * (N + 4)), smem_c = sizeof(float2) * (N + kEvTc * (N + 4));
  k_l2_strehl_rows<N><<<N / kEvTr, kEvRowThreads, smem_r, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_l2_strehl_cols<N><<<N / kEvTc, kEvColThreads, smem_c, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ddh
