// Cluster-per-stream kernels of the DDH-MBIR frame step (sm_103a).
//
// One thread-block cluster of C = N/16 CTAs (512 threads each) owns one stream's frame.
// CTA k holds, in shared memory,
//   * rows  rho = k + C l (l = 0..15) of the pupil plane: the frame y, phi, and a row buffer;
//   * the column slab x = 16 k .. 16 k + 15 of the image plane: a column buffer (one column
//     per warp, contiguous), r and s = E|g|^2;
//   * a row-major staging buffer that receives the row pass (later: two of the ICD's weight
//     arrays), the halo columns of r from the neighbouring slabs, and the halo pair weights.
// The 2-D DFT is a row pass (one warp per row), a transpose through distributed shared
// memory (16-byte remote stores of each row's 16-column segments into the column owner's
// staging buffer, and 16-byte stores of two-column chunks on the way back), and a column pass.
// Cluster barriers separate the frame's global dependencies:
//   B1 Normalize / tip-tilt statistics   B2 row IFFT -> columns   B3 r-init + column FFT -> rows
//   B4..B7 the four ICD colours (the last also guards shared memory until every reader is done).
// Each barrier is split into arrive and wait where local work can fill the gap: the r slab
// loads at B1, the slab's interior surrogate weights at B3, the next colour's interior pixels
// at B4..B6 (only work that reads no other CTA's pushes goes between the two).
// Per frame the kernel reads y (8 B/px), phi and r (4 B/px each) and writes phi and r.
// Everything before `grid_dep_wait` (frame TMA, twiddles, frame statistics) is independent of
// the previous frame, so under programmatic dependent launch it overlaps the previous frame's
// kernel on the same stream; the state (phi, r) is read only after the wait.
#include <cooperative_groups.h>

#include "ddh_device.cuh"
#include "ddh_kernels.cuh"

namespace cg = cooperative_groups;

namespace ddh {

template <int N>
struct StepLayout {
  static constexpr int C = N / kRowsPerCta;    // CTAs per cluster
  static constexpr int R = kRowsPerCta;        // local rows
  static constexpr int W = kRowsPerCta;        // slab columns
  static constexpr int CS = N + 1;             // padded column stride (floats / float2)
  static constexpr int RS = N + 2;             // row-buffer stride (float2): 16-byte aligned rows
  static constexpr size_t al(size_t v) { return (v + 127) & ~size_t(127); }
  static constexpr size_t tw = 0;
  static constexpr size_t rowbuf = al(tw + N * 8);
  static constexpr size_t colbuf = al(rowbuf + size_t(R) * RS * 8);
  static constexpr size_t ybuf = al(colbuf + size_t(W) * CS * 8);
  static constexpr size_t phib = al(ybuf + size_t(R) * N * 8);
  static constexpr size_t phin = al(phib + size_t(R) * N * 4);  // phi of row rho + 1
  static constexpr size_t rS = al(phin + size_t(R) * N * 4);
  static constexpr size_t sS = al(rS + size_t(W) * CS * 4);
  // row-major staging of the row pass for this slab: 16 columns (8 chunks of 2) per row
  // (it holds the SE and SW pair weights of the ICD once the column pass has read it)
  static constexpr size_t stage = al(sS + size_t(W) * CS * 4);
  static constexpr size_t stage_bytes =
      size_t(N) * 16 * 8 > size_t(2) * W * CS * 4 ? size_t(N) * 16 * 8 : size_t(2) * W * CS * 4;
  static constexpr size_t hl = al(stage + stage_bytes);          // r of the left slab's last column
  static constexpr size_t hr = al(hl + size_t(N) * 4);         // r of the right slab's first column
  static constexpr size_t halo = al(hr + size_t(N) * 4);       // 3 x N halo-pair weights
  static constexpr size_t red = al(halo + size_t(3) * N * 4);  // 16 warps x 8 floats
  static constexpr size_t pub = al(red + 16 * 8 * 4);         // 8 floats from each of the C CTAs
  static constexpr size_t glob = al(pub + 16 * 8 * 4);        // 8 combined floats
  static constexpr size_t mbar = al(glob + 8 * 4);
  static constexpr size_t total = al(mbar + 16);
};

// Rows are dealt to the cluster's CTAs cyclically in groups of G = 2^gs consecutive rows, so
// that a G x G phase tile stays inside one CTA: local row l of CTA k is global row
// G (k + C floor(l/G)) + (l mod G).
template <int C>
__device__ __forceinline__ int row_of(int k, int l, int gs) {
  return (((l >> gs) * C + k) << gs) + (l & ((1 << gs) - 1));
}
template <int C>
__device__ __forceinline__ int row_owner(int rho, int gs) { return (rho >> gs) % C; }
template <int C>
__device__ __forceinline__ int row_local(int rho, int gs) {
  return (((rho >> gs) / C) << gs) + (rho & ((1 << gs) - 1));
}

// Combine equal-size groups held one per lane (lanes with valid == false contribute nothing):
// overall mean = mean of the group means; M2 = sum_l (M2_l + n |m_l - mean|^2); plain sums for
// the rest.  Butterfly sums: every lane ends with the same, order-fixed result.
__device__ __forceinline__ void combine_equal_groups(float* v, bool valid, float n_group, float inv_groups) {
  float sx = warp_sum(valid ? v[0] : 0.f);
  float sy = warp_sum(valid ? v[1] : 0.f);
  const float mx = sx * inv_groups, my = sy * inv_groups;
  const float dx = v[0] - mx, dy = v[1] - my;
  const float q = warp_sum(valid ? fmaf(n_group, fmaf(dx, dx, dy * dy), v[2]) : 0.f);
  v[0] = mx;
  v[1] = my;
  v[2] = q;
#pragma unroll
  for (int j = 3; j < 8; ++j) v[j] = warp_sum(valid ? v[j] : 0.f);
}

template <int N, int V>
__global__ void __launch_bounds__(kThreads, 1) k_ddh_step(const __grid_constant__ StepBatch batch) {
  using L = StepLayout<N>;
  constexpr int C = L::C, R = L::R, W = L::W, CS = L::CS, RS = L::RS;
  extern __shared__ __align__(128) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int k = static_cast<int>(cluster.block_rank());
  const int sidx = blockIdx.x / C;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const KParams P = batch.prm[sidx];
  const FrameArgs A = batch.fa[sidx];

  float2* tw = reinterpret_cast<float2*>(smem + L::tw);
  float2* rowbuf = reinterpret_cast<float2*>(smem + L::rowbuf);
  float2* colbuf = reinterpret_cast<float2*>(smem + L::colbuf);
  float2* ybuf = reinterpret_cast<float2*>(smem + L::ybuf);
  float* phib = reinterpret_cast<float*>(smem + L::phib);
  float* phin = reinterpret_cast<float*>(smem + L::phin);
  float* rS = reinterpret_cast<float*>(smem + L::rS);
  float* sS = reinterpret_cast<float*>(smem + L::sS);
  float4* stage = reinterpret_cast<float4*>(smem + L::stage);
  float* hl = reinterpret_cast<float*>(smem + L::hl);
  float* hr = reinterpret_cast<float*>(smem + L::hr);
  float* halo = reinterpret_cast<float*>(smem + L::halo);
  float* red = reinterpret_cast<float*>(smem + L::red);
  float* pub = reinterpret_cast<float*>(smem + L::pub);
  float* glob = reinterpret_cast<float*>(smem + L::glob);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::mbar);
  const float cc = 0.5f * static_cast<float>(N - 1);
  const float invN = 1.f / static_cast<float>(N);

  // ---- phase 0: stage y rows by TMA and twiddles (independent of the previous frame) ------
  grid_dep_launch();  // the next frame's kernel may start its own prologue now
  if (tid == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (A.y_host) {
    // a frame in pinned host memory, read in place over the CPU-GPU link with 16-byte loads
    constexpr int NV = N / 2;  // float4 (two complex values) per row
    const float4* y4 = reinterpret_cast<const float4*>(A.y);
#pragma unroll 4
    for (int i = tid; i < R * NV; i += kThreads) {
      const int l = i / NV, xv = i - l * NV;
      reinterpret_cast<float4*>(ybuf + l * N)[xv] = y4[static_cast<size_t>(row_of<C>(k, l, P.g_shift)) * NV + xv];
    }
  } else if (tid == 0) {
    mbar_arrive_expect_tx(mbar, static_cast<uint32_t>(R * N * sizeof(float2)));
    const float2* y = batch.ytab != nullptr ? batch.ytab[batch.ytab_base + sidx] : A.y;
    for (int l = 0; l < R; ++l) {
      const int rho = row_of<C>(k, l, P.g_shift);
      tma_load_1d(ybuf + l * N, y + static_cast<size_t>(rho) * N, N * sizeof(float2), mbar);
    }
  }
  for (int i = tid; i < N; i += kThreads) tw[i] = batch.tw[i];
  // the grid's outer halo columns have no neighbour to fill them; the ICD still multiplies
  // them by a zero weight, which must not meet stale NaN or Inf bits in shared memory
  if (k == 0)
    for (int i = tid; i < N; i += kThreads) hl[i] = 0.f;
  if (k == C - 1)
    for (int i = tid; i < N; i += kThreads) hr[i] = 0.f;
  // bounded wait: on expiry the frame is dropped (flag carried into the B1 statistics)
  const bool loaded = A.y_host ? true : mbar_wait_bounded(mbar, 0, 1u << 22);
  __syncthreads();

  // ---- phase 1a: per-row statistics of the frame (Normalize, Eq. 4) ----------------------
  const int rho1 = row_of<C>(k, warp, P.g_shift);
  float2 mrow;
  float q = 0.f;
  {
    const float2* yr = ybuf + warp * N;
    float sre = 0.f, sim = 0.f;
    for (int x = lane; x < N; x += 32) { sre += yr[x].x; sim += yr[x].y; }
    sre = warp_sum(sre);
    sim = warp_sum(sim);
    mrow = make_float2(sre * invN, sim * invN);
    for (int x = lane; x < N; x += 32) q += c_abs2(c_sub(yr[x], mrow));
    q = warp_sum(q);
  }

  // ---- phase 0b: the state written by the previous frame: phi rows (r slab after B1's arrival)
  grid_dep_wait();
  // sigma^2 of this frame: the stream's running estimate when it is re-estimated (written by
  // the previous frame's post kernel), else the parameter
  const float nv = A.aux != nullptr ? A.aux[0] : P.noise_var;
  {
    // phi rows rho and rho + 1 (the latter for the y tip/tilt pairs), 16-byte vectors
    constexpr int NV4 = N / 4;
    const float4* src = reinterpret_cast<const float4*>(A.phi);
    for (int i = tid; i < R * NV4; i += kThreads) {
      const int l = i / NV4, xv = i - l * NV4;
      const int rho = row_of<C>(k, l, P.g_shift);
      reinterpret_cast<float4*>(phib)[i] = src[static_cast<size_t>(rho) * NV4 + xv];
      reinterpret_cast<float4*>(phin)[i] =
          rho + 1 < N ? src[static_cast<size_t>(rho + 1) * NV4 + xv] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  __syncthreads();

  // ---- phase 1b: tip/tilt sums (Sec. 4) ------------------------------------------------
  {
    const int l = warp, rho = rho1;
    float txs = 0.f, txc = 0.f, tys = 0.f, tyc = 0.f;
    if (P.tilt_mode) {
      const float* pr = phib + l * N;
      const int dy2 = ap_dist2(rho, N);
      const int dy2n = rho + 1 < N ? ap_dist2(rho + 1, N) : (1 << 30);
      for (int x = lane; x < N; x += 32) {
        const int dx2 = ap_dist2(x, N);
        if (dx2 + dy2 > P.ap_lim) continue;
        if (x + 1 < N && ap_dist2(x + 1, N) + dy2 <= P.ap_lim) {
          txs += wrap_pi(pr[x + 1] - pr[x]);
          txc += 1.f;
        }
        if (dx2 + dy2n <= P.ap_lim) {
          tys += wrap_pi(phin[l * N + x] - pr[x]);
          tyc += 1.f;
        }
      }
      txs = warp_sum(txs); txc = warp_sum(txc); tys = warp_sum(tys); tyc = warp_sum(tyc);
    }
    if (lane == 0) {
      float* o = red + warp * 8;
      o[0] = mrow.x; o[1] = mrow.y; o[2] = q; o[3] = txs; o[4] = txc; o[5] = tys; o[6] = tyc;
      o[7] = loaded ? 0.f : 1.f;
    }
  }
  __syncthreads();
  if (warp == 0) {  // the 16 rows of this CTA: equal groups of N samples
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = lane < 16 ? red[lane * 8 + j] : 0.f;
    combine_equal_groups(v, lane < 16, static_cast<float>(N), 1.f / 16.f);
    __syncwarp();
    if (lane < 8) red[lane] = v[lane];
  }
  __syncthreads();
  // push this CTA's partials into slot k of every CTA of the cluster (read locally after B1)
  if (tid < C) {
    const float4* srcv = reinterpret_cast<const float4*>(red);
    float4* dst = reinterpret_cast<float4*>(cluster.map_shared_rank(pub, tid) + 8 * k);
    dst[0] = srcv[0];
    dst[1] = srcv[1];
  }
  cluster_arrive();  // B1
  // the reflectance slab (W = 16 consecutive floats per row = 4 vectors) is first needed in
  // phase 3: its loads overlap the barrier
  for (int i = tid; i < N * (W / 4); i += kThreads) {
    const int rho = i / (W / 4), cv = i - rho * (W / 4);
    const float4 v = reinterpret_cast<const float4*>(A.r + static_cast<size_t>(rho) * N + W * k)[cv];
    rS[(4 * cv + 0) * CS + rho] = v.x;
    rS[(4 * cv + 1) * CS + rho] = v.y;
    rS[(4 * cv + 2) * CS + rho] = v.z;
    rS[(4 * cv + 3) * CS + rho] = v.w;
  }
  cluster_wait();  // B1
  if (warp == 0) {
    // lane q fetches CTA q's partials (C <= 32 remote loads in parallel), then lane 0
    // combines them in rank order, so every CTA derives bit-identical statistics
    float o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = 0.f;
    if (lane < C) {
      const float4* src = reinterpret_cast<const float4*>(pub + 8 * lane);
      const float4 a = src[0], b = src[1];
      o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
      o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    }
    combine_equal_groups(o, lane < C, static_cast<float>(R * N), 1.f / static_cast<float>(C));
    const float2 m_a = make_float2(o[0], o[1]);
    const float q_a = o[2], t0 = o[3], t1 = o[4], t2 = o[5], t3 = o[6], bad = o[7];
    if (lane == 0) {
    const float scale = sqrtf(static_cast<float>(N) * static_cast<float>(N) / q_a);
    const bool finite = isfinite(m_a.x) && isfinite(m_a.y) && isfinite(q_a) && q_a > 0.f && isfinite(scale);
    glob[0] = m_a.x;
    glob[1] = m_a.y;
    glob[2] = scale;
    glob[3] = (P.tilt_mode && t1 > 0.f) ? t0 / t1 : 0.f;
    glob[4] = (P.tilt_mode && t3 > 0.f) ? t2 / t3 : 0.f;
    glob[5] = (!finite || bad > 0.f) ? 1.f : 0.f;
    if (k == 0 && A.status != nullptr) {
      unsigned bits = 0;
      if (!finite) bits |= kStatusNonFinite;
      if (bad > 0.f) bits |= kStatusTimeout;
      if (bits) atomicOr(A.status, bits);
    }
    if (k == 0 && A.trace != nullptr) {
      float* st = A.trace + static_cast<size_t>(N) * N * 8;
      st[0] = m_a.x; st[1] = m_a.y; st[2] = scale; st[3] = glob[3]; st[4] = glob[4];
      st[5] = 0.f; st[6] = 0.f; st[7] = 0.f;
    }
    }
  }
  __syncthreads();
  const float2 ymean = make_float2(glob[0], glob[1]);
  const float scale = glob[2];
  const float tx = glob[3], ty = glob[4];
  if (glob[5] != 0.f) {  // uniform across the cluster: every CTA combined the same partials
    if (A.aux != nullptr && k == 0 && tid == 0) A.aux[1] = 0.f;  // the post kernel keeps the state
    // the state stays as it was, and so do its second destinations (rows of phi and the r slab
    // are in shared memory already)
    if (A.phi_copy != nullptr)
      for (int i = tid; i < R * N; i += kThreads) {
        const int l = i / N, x = i - l * N;
        A.phi_copy[static_cast<size_t>(row_of<C>(k, l, P.g_shift)) * N + x] = phib[i];
      }
    if (A.r_copy != nullptr)
      for (int i = tid; i < N * W; i += kThreads) {
        const int rho = i / W, cl = i - rho * W;
        A.r_copy[static_cast<size_t>(rho) * N + W * k + cl] = rS[cl * CS + rho];
      }
    cluster.sync();
    return;
  }

  for (int it = 0; it < P.n_k; ++it) {
    const bool first = (it == 0);
    float* trace = first ? A.trace : nullptr;
    const bool aux_out = A.aux != nullptr && it == P.n_k - 1;  // side outputs of the last iteration
    // ---- phase 2: back-projection prologue a e^{-j phi} y~ and row IFFT (aperture rows) --
    {
      const int l = warp, rho = row_of<C>(k, l, P.g_shift);
      const int dy2 = ap_dist2(rho, N);
      float2* rb = rowbuf + l * RS;
      float* pr = phib + l * N;
      const float2* yr = ybuf + l * N;
      if (dy2 <= P.ap_lim) {
        const float tyr = ty * (static_cast<float>(rho) - cc);
        for (int x = lane; x < N; x += 32) {
          if (ap_dist2(x, N) + dy2 <= P.ap_lim) {
            float ph = pr[x];
            if (first && P.tilt_mode) ph = wrap_pi(ph - fmaf(tx, static_cast<float>(x) - cc, tyr));
            pr[x] = ph;
            const float2 yt = c_scale(c_sub(yr[x], ymean), scale);
            float sn, cs;
            sincosf(ph, &sn, &cs);
            rb[swz(x)] = make_float2(fmaf(yt.x, cs, yt.y * sn), fmaf(yt.y, cs, -yt.x * sn));
          } else {
            rb[swz(x)] = make_float2(0.f, 0.f);
            pr[x] = 0.f;
          }
        }
        __syncwarp();
        fft_row<N, +1, V>(rb, tw, lane);
        // transpose: CTA j receives columns 16 j .. 16 j + 15 of this row as 8 chunks of two
        // (16-byte remote stores), chunk m at slot m ^ (rho & 7) of stage row rho, its two
        // values swapped when bit 3 of rho is set (the column reads below are conflict-free)
        const int sw = rho & 7, sp = (rho >> 3) & 1;
        for (int g = lane; g < N / 2; g += 32) {
          const int j = g >> 3, m = g & 7;
          const float2 a = rb[16 * j + ((2 * m) ^ j)];      // swz(16 j + o) = 16 j + (o ^ j)
          const float2 b = rb[16 * j + ((2 * m + 1) ^ j)];
          const float4 v = sp ? make_float4(b.x, b.y, a.x, a.y) : make_float4(a.x, a.y, b.x, b.y);
          cluster.map_shared_rank(stage, j)[rho * 8 + (m ^ sw)] = v;
        }
      } else {
        for (int x = lane; x < N; x += 32) pr[x] = 0.f;
      }
    }
    cluster.sync();  // B2
    // ---- phase 3: column IFFT, r-init (Eq. 3) + E-step, column FFT of mu, scatter ---------
    {
      const int cl = warp;
      float2* cb = colbuf + cl * CS;
      {
        // the first IFFT pass gathers the column straight from the staging buffer (rows
        // outside the aperture are zero and were not sent)
        const float2* st2 = reinterpret_cast<const float2*>(stage);
        const int ap_lim = P.ap_lim;
        auto gather = [st2, cl, ap_lim](int rho) {
          return ap_dist2(rho, N) <= ap_lim
                     ? st2[rho * 16 + 2 * ((cl >> 1) ^ (rho & 7)) + ((cl & 1) ^ ((rho >> 3) & 1))]
                     : make_float2(0.f, 0.f);
        };
        fft_row_from<N, +1, V>(cb, tw, lane, gather);
      }
      float csum = 0.f;  // sum of the posterior variances C = sigma^2 w (side output)
      for (int rho = lane; rho < N; rho += 32) {
        const float2 b = c_scale(cb[swz(rho)], invN);
        const float rp = rS[cl * CS + rho];
        const float ri = first ? fmaxf(fmaf(P.lam1, rp, P.lam_alpha * c_abs2(b)), P.r_floor) : rp;
        const float wgt = ri * hw_rcp(ri + nv);
        const float2 mu = c_scale(b, wgt);
        const float s = fmaf(nv, wgt, c_abs2(mu));
        if (aux_out) csum += nv * wgt;
        cb[swz(rho)] = mu;
        rS[cl * CS + rho] = ri;
        sS[cl * CS + rho] = s;
        // slab-edge values go to the neighbouring slabs' halo columns (read after B3)
        if (cl == 0 && k > 0) cluster.map_shared_rank(hr, k - 1)[rho] = ri;
        if (cl == W - 1 && k < C - 1) cluster.map_shared_rank(hl, k + 1)[rho] = ri;
        if (trace != nullptr) {
          const size_t gi = static_cast<size_t>(rho) * N + W * k + cl;
          const size_t M = static_cast<size_t>(N) * N;
          reinterpret_cast<float2*>(trace)[gi] = b;
          reinterpret_cast<float2*>(trace)[M + gi] = mu;
          trace[6 * M + gi] = ri;
          trace[7 * M + gi] = s;
        }
      }
      if (aux_out) {
        csum = warp_sum(csum);
        if (lane == 0) red[warp] = csum;
      }
      __syncwarp();
      fft_row<N, -1, V>(cb, tw, lane);
    }
    __syncthreads();  // every column of the slab is transformed
    // transpose back: the 16 slab values of aperture row rho go to the row owner as 8 chunks
    // of two (16-byte remote stores); chunk m covers positions 16 k + 2m, 16 k + 2m + 1 of the
    // owner's swizzled row, which hold columns (2m) ^ k and (2m + 1) ^ k of this slab
    for (int f = tid; f < N * 8; f += kThreads) {
      const int rho = f >> 3, m = f & 7;
      if (ap_dist2(rho, N) > P.ap_lim) continue;
      const float2 a = colbuf[((2 * m) ^ k) * CS + swz(rho)];
      const float2 b = colbuf[((2 * m + 1) ^ k) * CS + swz(rho)];
      float2* row = cluster.map_shared_rank(rowbuf, row_owner<C>(rho, P.g_shift)) + row_local<C>(rho, P.g_shift) * RS;
      reinterpret_cast<float4*>(row + W * k)[m] = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();  // the column buffer's last readers are done: it now takes weights
    cluster_arrive();  // B3
    // Surrogate weights beta_ij = b_ij rho'(D)/D at the entry values (r-init), once per pixel
    // pair: E, S, SE, SW pairs of every slab pixel (E, S in the column buffer, SE, SW in the
    // staging buffer, both idle now), and the three pairs that cross into the left/right slabs
    // from this side (W, NW at cl = 0; NE at cl = W-1).  A pair shared by two CTAs gets the same
    // value on both sides (|D| symmetric).  The slab's interior pairs are formed while the
    // cluster barrier completes; the edge columns and the halo pairs read the neighbours'
    // pushed r-init columns after it.
    {
      float* bE = reinterpret_cast<float*>(colbuf);
      float* bS = bE + W * CS;
      float* bSE = reinterpret_cast<float*>(stage);
      float* bSW = bSE + W * CS;
      // before colour 0 the slab holds r-init, and hl / hr hold the neighbours' edge columns
      auto wgt = [&](float d) { return prior_weight_fast(d, P.w0, P.inv_tsig, P.q_minus_p, P.q_over_p); };
      // every load of a batch precedes its stores (the weight arrays alias other buffers, so
      // a load after a store could not be moved above it), which keeps 4 pixels x 4 weights
      // of MUFU work in flight per thread
      constexpr int kPx = W * N / kThreads;  // pixels per thread (N / 32)
      constexpr int kB = kPx < 4 ? kPx : 4;
      // edge == false: the pixels of columns 1 .. W-2, whose pairs lie inside this slab;
      // edge == true: columns 0 and W-1, whose pairs reach the neighbours' pushed columns
      auto pair_weights = [&](bool edge) {
#pragma unroll
      for (int u0 = 0; u0 < kPx; u0 += kB) {
        float dd[kB][4];
        bool ok[kB][4];
        int oo[kB];
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          const int i = tid + kThreads * (u0 + b);
          const int cl = i / N, rho = i - cl * N;
          const int x = W * k + cl;
          const int o = cl * CS + rho;
          oo[b] = ((cl == 0 || cl == W - 1) == edge) ? o : -1;
          if (oo[b] < 0) {
#pragma unroll
            for (int e = 0; e < 4; ++e) { dd[b][e] = 0.f; ok[b][e] = false; }
            continue;
          }
          const bool dn = rho + 1 < N;
          const float r0i = rS[o];
          const float rE = cl + 1 < W ? rS[o + CS] : hr[rho];
          const float rSo = dn ? rS[o + 1] : 0.f;
          const float rSE = !dn ? 0.f : (cl + 1 < W ? rS[o + CS + 1] : hr[rho + 1]);
          const float rSW = !dn ? 0.f : (cl > 0 ? rS[o - CS + 1] : hl[rho + 1]);
          dd[b][0] = r0i - rE;  dd[b][1] = r0i - rSo;  dd[b][2] = r0i - rSE;  dd[b][3] = r0i - rSW;
          ok[b][0] = x + 1 < N;  ok[b][1] = dn;  ok[b][2] = x + 1 < N && dn;  ok[b][3] = x > 0 && dn;
        }
        float ww[kB][4];
#pragma unroll
        for (int b = 0; b < kB; ++b) {
#pragma unroll
          for (int e = 0; e < 4; ++e) ww[b][e] = ok[b][e] ? (e < 2 ? kBnn : kBdiag) * wgt(dd[b][e]) : 0.f;
        }
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          if (oo[b] < 0) continue;
          bE[oo[b]] = ww[b][0];
          bS[oo[b]] = ww[b][1];
          bSE[oo[b]] = ww[b][2];
          bSW[oo[b]] = ww[b][3];
        }
      }
      };
      pair_weights(false);
      cluster_wait();  // B3: neighbours' row segments and edge columns have arrived
      pair_weights(true);
      for (int rho = tid; rho < N; rho += kThreads) {
        // hW: pair (rho, x0-1)-(rho, x0); hNW: (rho-1, x0-1)-(rho, x0); hNE: (rho-1, x1+1)-(rho, x1)
        const float a0 = rS[rho], a1 = rS[(W - 1) * CS + rho];
        halo[rho] = k > 0 ? kBnn * wgt(a0 - hl[rho]) : 0.f;
        halo[N + rho] = (k > 0 && rho > 0) ? kBdiag * wgt(a0 - hl[rho - 1]) : 0.f;
        halo[2 * N + rho] = (k < C - 1 && rho > 0) ? kBdiag * wgt(a1 - hr[rho - 1]) : 0.f;
      }
    }
    // ---- phase 4: row FFT of mu (aperture rows) and phase M-step ------------------------
    // v = a y~ conj(z) per pixel (summed over the G x G tile when G > 1); phi = angle(v).
    {
      const int gs = P.g_shift, G = 1 << gs;
      const int l = warp, rho = row_of<C>(k, l, gs);
      const int dy2 = ap_dist2(rho, N);
      const bool row_ap = dy2 <= P.ap_lim;
      float2* rb = rowbuf + l * RS;
      const float2* yr = ybuf + l * N;
      if (row_ap) fft_row<N, -1, V>(rb, tw, lane);
      for (int x = lane; x < N; x += 32) {
        float2 v = make_float2(0.f, 0.f);
        float e = 0.f;  // a (|y~|^2 + |z|^2) (side output)
        if (row_ap && ap_dist2(x, N) + dy2 <= P.ap_lim) {
          const float2 z = c_scale(rb[swz(x)], invN);
          const float2 yt = c_scale(c_sub(yr[x], ymean), scale);
          v = make_float2(fmaf(yt.x, z.x, yt.y * z.y), fmaf(yt.y, z.x, -yt.x * z.y));
          if (aux_out) e = c_abs2(yt) + c_abs2(z);
          if (trace != nullptr) {
            const size_t M = static_cast<size_t>(N) * N;
            reinterpret_cast<float2*>(trace)[2 * M + static_cast<size_t>(rho) * N + x] = z;
          }
        }
        for (int o = 1; o < G; o <<= 1) {  // sum over the G consecutive x of the tile
          v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
          v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
          if (aux_out) e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        rb[swz(x)] = v;
        if (aux_out) phin[l * N + x] = e;  // phin (the tip/tilt rows) is free after phase 1
      }
    }
    if (P.g_shift > 0) __syncthreads();  // tile rows are other warps of this CTA
    {
      const int gs = P.g_shift, G = 1 << gs;
      const int l = warp, rho = row_of<C>(k, l, gs);
      const int dy2 = ap_dist2(rho, N);
      const int l0 = l & ~(G - 1);
      float* pr = phib + l * N;
      float* phi_out = A.phi + static_cast<size_t>(rho) * N;
      for (int x = lane; x < N; x += 32) {
        float out = 0.f;
        if (dy2 <= P.ap_lim && ap_dist2(x, N) + dy2 <= P.ap_lim) {
          float2 v = rowbuf[l0 * RS + swz(x)];
          for (int j = 1; j < G; ++j) v = c_add(v, rowbuf[(l0 + j) * RS + swz(x)]);
          out = (v.x != 0.f || v.y != 0.f) ? atan2f(v.y, v.x) : pr[x];
          pr[x] = out;
        }
        phi_out[x] = out;
        if (A.phi_copy != nullptr && it == P.n_k - 1) A.phi_copy[static_cast<size_t>(rho) * N + x] = out;
      }
    }
    __syncthreads();  // the surrogate weights (formed around B3) and phase 4 are complete
    if (aux_out) {
      // Side outputs for the post kernel, per G x G tile of this CTA's rows: the tile sums
      // v_t (as in the phase step) and E_t.  With the phase prior they go to the tile grid;
      // otherwise the tile phase is angle(v_t) and the pupil residual sum |y~ - e^{j phi} z|^2
      // over the tile is E_t - 2 |v_t|, summed here.  Then this CTA's two partial sums.
      const int gs = P.g_shift, G = 1 << gs, NT = N >> gs;
      float res = 0.f;
      for (int t = tid; t < (R >> gs) * NT; t += kThreads) {
        const int tl = t / NT, tx = t - tl * NT;
        const int l0 = tl << gs, x0 = tx << gs;
        float2 v = rowbuf[l0 * RS + swz(x0)];
        float e = phin[l0 * N + x0];
        for (int j = 1; j < G; ++j) {
          v = c_add(v, rowbuf[(l0 + j) * RS + swz(x0)]);
          e += phin[(l0 + j) * N + x0];
        }
        if (A.aux_tiles) {
          const int T = row_of<C>(k, l0, gs) >> gs;
          if (tile_in_pupil(T, tx, gs, N, P.ap_lim))
            reinterpret_cast<float4*>(A.aux + kAuxTiles)[T * NT + tx] = make_float4(v.x, v.y, e, 0.f);
        } else {
          res += e - 2.f * sqrtf(fmaf(v.x, v.x, v.y * v.y));
        }
      }
      res = warp_sum(res);
      if (lane == 0) red[16 + warp] = res;
      __syncthreads();
      if (tid == 0) {
        float sr = 0.f, sc = 0.f;
        for (int w = 0; w < 16; ++w) {
          sr += red[16 + w];
          sc += red[w];
        }
        A.aux[kAuxPart + 2 * k] = sr;
        A.aux[kAuxPart + 2 * k + 1] = sc;
        if (k == 0) A.aux[1] = 1.f;
      }
    }
    // ---- phase 5: r M-step, 4-colour ICD sweep on the q-GGMRF surrogate ------------------
    {
      float* bE = reinterpret_cast<float*>(colbuf);
      float* bS = bE + W * CS;
      float* bSE = reinterpret_cast<float*>(stage);
      float* bSW = bSE + W * CS;
      float* hr_left = k > 0 ? cluster.map_shared_rank(hr, k - 1) : hr;
      float* hl_right = k < C - 1 ? cluster.map_shared_rank(hl, k + 1) : hl;
      // One colour in two passes: its interior pixels read only this slab, its edge column
      // (cl = 0 for cx = 0, cl = W-1 for cx = 1) also reads the halo values that the
      // neighbouring slabs push.  The interior of colour c runs between this CTA's arrival at
      // the previous colour's cluster barrier and its wait there, so that the barrier's latency
      // is hidden; the edge column runs after the wait and pushes its own values.
      auto colour_pass = [&](int c, bool edge) {
        const int cx = c & 1, cy = c >> 1;  // colours (0,0), (1,0), (0,1), (1,1)
        // the pixels of one colour are not neighbours of each other: every thread loads the
        // inputs of all its pixels, solves, then stores (kCp = 4N / 512 pixels per thread)
        constexpr int kCp = (4 * N + kThreads - 1) / kThreads;
        float Wv[kCp], Cv[kCp], sv[kCp], rv[kCp];
        int ov[kCp], cv[kCp], hv[kCp];
#pragma unroll
        for (int u = 0; u < kCp; ++u) {
          const int idx = tid + kThreads * u;
          ov[u] = -1;
          if (4 * N % kThreads != 0 && idx >= 4 * N) continue;
          const int j = idx % (N / 2), ci = idx / (N / 2);
          const int cl = cx + 2 * ci, rho = cy + 2 * j;
          if ((cl == 0 || cl == W - 1) != edge) continue;
          const int o = cl * CS + rho;
          const bool up = rho > 0, dn = rho + 1 < N;
          // neighbour values: current r (earlier colours already updated)
          const float rW = cl > 0 ? rS[o - CS] : hl[rho];
          const float rE = cl + 1 < W ? rS[o + CS] : hr[rho];
          const float rN = up ? rS[o - 1] : 0.f;
          const float rSo = dn ? rS[o + 1] : 0.f;
          const float rNW = !up ? 0.f : (cl > 0 ? rS[o - CS - 1] : hl[rho - 1]);
          const float rNE = !up ? 0.f : (cl + 1 < W ? rS[o + CS - 1] : hr[rho - 1]);
          const float rSW = !dn ? 0.f : (cl > 0 ? rS[o - CS + 1] : hl[rho + 1]);
          const float rSE = !dn ? 0.f : (cl + 1 < W ? rS[o + CS + 1] : hr[rho + 1]);
          // pair weights (zero where the neighbour is off the grid)
          const float wE = bE[o], wS = bS[o], wSE = bSE[o], wSW = bSW[o];
          const float wW = cl > 0 ? bE[o - CS] : halo[rho];
          const float wN = up ? bS[o - 1] : 0.f;
          const float wNW = !up ? 0.f : (cl > 0 ? bSE[o - CS - 1] : halo[N + rho]);
          const float wNE = !up ? 0.f : (cl + 1 < W ? bSW[o + CS - 1] : halo[2 * N + rho]);
          Wv[u] = ((wN + wS) + (wW + wE)) + ((wNW + wNE) + (wSW + wSE));
          float Csum = wN * rN;
          Csum = fmaf(wS, rSo, Csum);
          Csum = fmaf(wW, rW, Csum);
          Csum = fmaf(wE, rE, Csum);
          Csum = fmaf(wNW, rNW, Csum);
          Csum = fmaf(wNE, rNE, Csum);
          Csum = fmaf(wSW, rSW, Csum);
          Csum = fmaf(wSE, rSE, Csum);
          Cv[u] = Csum;
          sv[u] = sS[o];
          rv[u] = rS[o];
          ov[u] = o;
          cv[u] = cl;
          hv[u] = rho;
        }
#pragma unroll
        for (int u = 0; u < kCp; ++u) {
          if (ov[u] < 0) continue;
          const float rn = fmaxf(icd_root_from(Wv[u], Cv[u], sv[u], rv[u]), P.r_floor);
          rS[ov[u]] = rn;
          // edge pixels of this colour are read by the neighbouring slab in the next colours
          if (cv[u] == 0 && k > 0) hr_left[hv[u]] = rn;
          if (cv[u] == W - 1 && k < C - 1) hl_right[hv[u]] = rn;
        }
      };
      for (int c = 0; c < 4; ++c) {
        colour_pass(c, false);
        if (c > 0) cluster_wait();  // B4..B6: the previous colour's halo pushes are visible
        colour_pass(c, true);
        __syncthreads();            // this colour's slab updates before the next interior pass
        cluster_arrive();           // B4..B7
      }
      cluster_wait();  // B7 (also guards shared memory until every remote reader is done)
    }
  }
  // ---- write the reflectance slab back (row-major N x N) ---------------------------------
  for (int i = tid; i < N * W; i += kThreads) {
    const int rho = i / W, cl = i - rho * W;
    const float v = rS[cl * CS + rho];
    A.r[static_cast<size_t>(rho) * N + W * k + cl] = v;
    if (A.r_copy != nullptr) A.r_copy[static_cast<size_t>(rho) * N + W * k + cl] = v;
  }
}

// Strehl ratio (Sec. 5.B): max |F^H(a e^{j(phi_true - phi_est)})|^2 / max |F^H a|^2.
template <int N>
__global__ void __launch_bounds__(kThreads, 1) k_strehl(const __grid_constant__ StrehlArgs a) {
  using L = StepLayout<N>;
  constexpr int C = L::C, W = L::W, CS = L::CS;
  extern __shared__ __align__(128) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int k = static_cast<int>(cluster.block_rank());
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* tw = reinterpret_cast<float2*>(smem + L::tw);
  float2* rowbuf = reinterpret_cast<float2*>(smem + L::rowbuf);
  float2* colbuf = reinterpret_cast<float2*>(smem + L::colbuf);
  float* red = reinterpret_cast<float*>(smem + L::red);
  float* pub = reinterpret_cast<float*>(smem + L::pub);
  for (int i = tid; i < N; i += kThreads) tw[i] = a.tw[i];
  for (int i = tid; i < W * CS; i += kThreads) colbuf[i] = make_float2(0.f, 0.f);
  __syncthreads();
  cluster.sync();
  {
    const int l = warp, rho = k + C * l;
    const int dy2 = ap_dist2(rho, N);
    if (dy2 <= a.ap_lim) {
      float2* rb = rowbuf + l * N;
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
      for (int x = lane; x < N; x += 32) cluster.map_shared_rank(colbuf, x / W)[(x % W) * CS + swz(rho)] = rb[swz(x)];
    }
  }
  cluster.sync();
  float m = 0.f;
  {
    float2* cb = colbuf + warp * CS;
    fft_row<N, +1>(cb, tw, lane);
    for (int rho = lane; rho < N; rho += 32) m = fmaxf(m, c_abs2(cb[swz(rho)]));
    m = warp_max(m);
  }
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (tid == 0) {
    float mm = red[0];
    for (int w = 1; w < 16; ++w) mm = fmaxf(mm, red[w]);
    pub[0] = mm;
  }
  cluster.sync();
  if (k == 0 && tid == 0) {
    float mm = 0.f;
    for (int q = 0; q < C; ++q) mm = fmaxf(mm, cluster.map_shared_rank(pub, q)[0]);
    // unscaled transforms: |F^H u|^2 = |v|^2 / N^2 and max |F^H a|^2 = (sum a)^2 / N^2
    a.out[0] = mm * a.inv_ap_count2;
  }
  cluster.sync();
}

// Unitary 2-D DFT (or inverse) of one N x N image; in and out may alias.
template <int N>
__global__ void __launch_bounds__(kThreads, 1) k_fft2(const __grid_constant__ Fft2Args a) {
  using L = StepLayout<N>;
  constexpr int C = L::C, R = L::R, W = L::W, CS = L::CS;
  extern __shared__ __align__(128) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int k = static_cast<int>(cluster.block_rank());
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* tw = reinterpret_cast<float2*>(smem + L::tw);
  float2* rowbuf = reinterpret_cast<float2*>(smem + L::rowbuf);
  float2* colbuf = reinterpret_cast<float2*>(smem + L::colbuf);
  grid_dep_launch();
  for (int i = tid; i < N; i += kThreads) tw[i] = a.tw[i];
  grid_dep_wait();  // `in` may be the previous kernel's output
  {
    // every load of a thread before its first store into the row buffer
    constexpr int PER = R * N / kThreads;
    float2 v[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid + kThreads * j, l = i / N, x = i - l * N;
      v[j] = a.in[static_cast<size_t>(k + C * l) * N + x];
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid + kThreads * j, l = i / N, x = i - l * N;
      rowbuf[l * N + swz(x)] = v[j];
    }
  }
  __syncthreads();
  cluster.sync();  // every read of `in` precedes every write of `out`
  {
    const int l = warp, rho = k + C * l;
    float2* rb = rowbuf + l * N;
    if (a.inverse) fft_row<N, +1>(rb, tw, lane);
    else fft_row<N, -1>(rb, tw, lane);
    for (int x = lane; x < N; x += 32) cluster.map_shared_rank(colbuf, x / W)[(x % W) * CS + swz(rho)] = rb[swz(x)];
  }
  cluster.sync();
  {
    float2* cb = colbuf + warp * CS;
    if (a.inverse) fft_row<N, +1>(cb, tw, lane);
    else fft_row<N, -1>(cb, tw, lane);
  }
  __syncthreads();
  const float invN = 1.f / static_cast<float>(N);
  for (int i = tid; i < N * W; i += kThreads) {
    const int rho = i / W, cl = i - rho * W;
    a.out[static_cast<size_t>(rho) * N + W * k + cl] = c_scale(colbuf[cl * CS + swz(rho)], invN);
  }
  cluster.sync();
}

// ------------------------------------------------------------------------------ launchers
template <typename Kern, typename Arg>
static cudaError_t launch_cluster(Kern kern, int c, int clusters, size_t smem, cudaStream_t st, const Arg& arg,
                                  bool pdl = false) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(c * clusters), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(c);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kern, arg);
}

template <int N, int V>
static cudaError_t configure_nv(int* max_active) {
  using L = StepLayout<N>;
  const void* f = reinterpret_cast<const void*>(k_ddh_step<N, V>);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L::total));
  if (e == cudaSuccess && L::C > 8) e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess || max_active == nullptr) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L::C, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = L::total;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L::C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(max_active, f, &cfg);
}

template <int N>
static cudaError_t configure_n(int* max_active) {
  using L = StepLayout<N>;
  const void* kerns[2] = {reinterpret_cast<const void*>(k_strehl<N>), reinterpret_cast<const void*>(k_fft2<N>)};
  for (const void* f : kerns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L::total));
    if (e != cudaSuccess) return e;
    if (L::C > 8) {
      e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
  }
  cudaError_t e = configure_nv<N, 0>(max_active);
  if (e != cudaSuccess) return e;
  if constexpr (FftSchedules<N>::count > 1) { e = configure_nv<N, 1>(nullptr); if (e != cudaSuccess) return e; }
  if constexpr (FftSchedules<N>::count > 2) { e = configure_nv<N, 2>(nullptr); if (e != cudaSuccess) return e; }
  return cudaSuccess;
}

cudaError_t configure(int n, int* max_active) {
  switch (n) {
    case 32: return configure_n<32>(max_active);
    case 64: return configure_n<64>(max_active);
    case 128: return configure_n<128>(max_active);
    case 256: return configure_n<256>(max_active);
    default: return cudaErrorInvalidValue;
  }
}

int schedule_count(int n) {
  switch (n) {
    case 512: return FftSchedules<512>::count;
    case 32: return FftSchedules<32>::count;
    case 64: return FftSchedules<64>::count;
    case 128: return FftSchedules<128>::count;
    case 256: return FftSchedules<256>::count;
    default: return 0;
  }
}

size_t step_smem_bytes(int n) {
  switch (n) {
    case 32: return StepLayout<32>::total;
    case 64: return StepLayout<64>::total;
    case 128: return StepLayout<128>::total;
    case 256: return StepLayout<256>::total;
    default: return 0;
  }
}

template <int N>
static cudaError_t launch_step_n(int v, const StepBatch& b, cudaStream_t st, bool pdl) {
  using L = StepLayout<N>;
  if (v == 0) return launch_cluster(k_ddh_step<N, 0>, L::C, b.count, L::total, st, b, pdl);
  if constexpr (FftSchedules<N>::count > 1) {
    if (v == 1) return launch_cluster(k_ddh_step<N, 1>, L::C, b.count, L::total, st, b, pdl);
  }
  if constexpr (FftSchedules<N>::count > 2) {
    if (v == 2) return launch_cluster(k_ddh_step<N, 2>, L::C, b.count, L::total, st, b, pdl);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step(int n, int v, const StepBatch& b, cudaStream_t st, bool pdl) {
  switch (n) {
    case 32: return launch_step_n<32>(v, b, st, pdl);
    case 64: return launch_step_n<64>(v, b, st, pdl);
    case 128: return launch_step_n<128>(v, b, st, pdl);
    case 256: return launch_step_n<256>(v, b, st, pdl);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_strehl(int n, const StrehlArgs& a, cudaStream_t st) {
  switch (n) {
    case 32: return launch_cluster(k_strehl<32>, StepLayout<32>::C, 1, StepLayout<32>::total, st, a);
    case 64: return launch_cluster(k_strehl<64>, StepLayout<64>::C, 1, StepLayout<64>::total, st, a);
    case 128: return launch_cluster(k_strehl<128>, StepLayout<128>::C, 1, StepLayout<128>::total, st, a);
    case 256: return launch_cluster(k_strehl<256>, StepLayout<256>::C, 1, StepLayout<256>::total, st, a);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fft2(int n, const Fft2Args& a, cudaStream_t st) {
  switch (n) {
    case 32: return launch_cluster(k_fft2<32>, StepLayout<32>::C, 1, StepLayout<32>::total, st, a, true);
    case 64: return launch_cluster(k_fft2<64>, StepLayout<64>::C, 1, StepLayout<64>::total, st, a, true);
    case 128: return launch_cluster(k_fft2<128>, StepLayout<128>::C, 1, StepLayout<128>::total, st, a, true);
    case 256: return launch_cluster(k_fft2<256>, StepLayout<256>::C, 1, StepLayout<256>::total, st, a, true);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ddh
