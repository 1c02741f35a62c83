// L2-staged frame step for grids whose working set exceeds a thread-block cluster's shared
// memory (512 x 512: about 10 MB per stream).  The same stages as the cluster kernel, as a
// sequence of batched kernels (blockIdx.y = stream of the batch) over per-stream global
// scratch that stays resident in the 129 MB L2 between stages:
//   s1 row statistics (Normalize, Eq. 4) and tip/tilt sums        (16 rows per block)
//   s2 combine; RemoveTipTilt, prologue a e^{-j phi'} y~, row IFFT; transposed store (8 rows)
//   s3 column IFFT, r-init (Eq. 3) + E-step, column FFT of mu; transposed store (8 cols/block)
//   s4 row FFT and phase M-step (tile sums when the phase is tiled)  (8 rows per block)
//   s5 surrogate weights of the E, S, SE, SW pairs; s6 one ICD colour (launched 4 times)
// Each 1-D DFT is the warp-per-row shared-memory Stockham FFT of the cluster kernel; the
// transposes go through an 8-row or 8-column shared-memory tile, so that global accesses are
// 32- or 64-byte runs.
// The stages are launched with programmatic stream serialization: each kernel lets its
// successor launch as soon as all its blocks run, and waits (`griddepcontrol.wait`, every
// thread, before any read of another stage's output and before any early return) until its
// predecessor has completed, so that the completion of one stage implies that of all earlier ones.
#include <utility>

#include "ddh_device.cuh"
#include "ddh_kernels.cuh"

namespace ddh {

namespace {

constexpr int kT = 16;  // rows per statistics block
constexpr int kTc = 8;  // columns per column-pass block (one warp per column)
constexpr int kColThreads = 32 * kTc;
constexpr int kTr = 8;  // rows per row-pass block (one warp per row)
constexpr int kRowThreads = 32 * kTr;

__device__ __forceinline__ bool frame_dropped(const L2Stream& S) { return *S.flag != 0; }

// ---- s1: per-row statistics and tip/tilt partial sums ---------------------------------------
// One block of kT rows of stream `sid` (block `bx`): each warp takes whole rows (one row per
// warp with 512 threads, two with 256); thread 0 combines the rows in row order.
template <int N>
__device__ __forceinline__ void l2_stage_stats(const L2Batch& b, int sid, int bx) {
  const L2Stream& S = b.st[sid];
  const KParams& P = b.prm[sid];
  const float2* y = b.ytab != nullptr ? b.ytab[b.ytab_base + sid] : S.y;
  __shared__ float red[16][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int lr = warp; lr < kT; lr += static_cast<int>(blockDim.x >> 5)) {
    const int rho = kT * bx + lr;
    constexpr int PER = N / 32;
    float2 v[PER];
    float sre = 0.f, sim = 0.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      v[j] = y[static_cast<size_t>(rho) * N + lane + 32 * j];
      sre += v[j].x;
      sim += v[j].y;
    }
    sre = warp_sum(sre);
    sim = warp_sum(sim);
    const float invN = 1.f / static_cast<float>(N);
    const float2 m = make_float2(sre * invN, sim * invN);
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) q += c_abs2(c_sub(v[j], m));
    q = warp_sum(q);
    // the frame's statistics above do not depend on the previous stage; phi and the
    // statistics buffers below do
    grid_dep_wait();
    float txs = 0.f, txc = 0.f, tys = 0.f, tyc = 0.f;
    if (P.tilt_mode) {
      const float* pr = S.phi + static_cast<size_t>(rho) * N;
      const int dy2 = ap_dist2(rho, N);
      const int dy2n = rho + 1 < N ? ap_dist2(rho + 1, N) : (1 << 30);
      for (int x = lane; x < N; x += 32) {
        const int dx2 = ap_dist2(x, N);
        if (dx2 + dy2 > P.ap_lim) continue;
        if (x + 1 < N && ap_dist2(x + 1, N) + dy2 <= P.ap_lim) { txs += wrap_pi(pr[x + 1] - pr[x]); txc += 1.f; }
        if (dx2 + dy2n <= P.ap_lim) { tys += wrap_pi(pr[x + N] - pr[x]); tyc += 1.f; }
      }
      txs = warp_sum(txs); txc = warp_sum(txc); tys = warp_sum(tys); tyc = warp_sum(tyc);
    }
    if (lane == 0) {
      red[lr][0] = m.x; red[lr][1] = m.y; red[lr][2] = q;
      red[lr][3] = txs; red[lr][4] = txc; red[lr][5] = tys; red[lr][6] = tyc;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float n_a = static_cast<float>(N), q_a = red[0][2];
    float2 m_a = make_float2(red[0][0], red[0][1]);
    float t0 = red[0][3], t1 = red[0][4], t2 = red[0][5], t3 = red[0][6];
    for (int w = 1; w < kT; ++w) {
      const float n_b = static_cast<float>(N);
      const float nn = n_a + n_b;
      const float2 d = make_float2(red[w][0] - m_a.x, red[w][1] - m_a.y);
      const float f = n_b / nn;
      m_a = make_float2(fmaf(d.x, f, m_a.x), fmaf(d.y, f, m_a.y));
      q_a = q_a + red[w][2] + c_abs2(d) * (n_a * f);
      n_a = nn;
      t0 += red[w][3]; t1 += red[w][4]; t2 += red[w][5]; t3 += red[w][6];
    }
    float* o = S.part + 8 * bx;
    o[0] = m_a.x; o[1] = m_a.y; o[2] = q_a; o[3] = t0; o[4] = t1; o[5] = t2; o[6] = t3; o[7] = 0.f;
    if (bx == 0) {
      *S.flag = 0;
      if (b.aux[sid] != nullptr) b.aux[sid][1] = 0.f;  // set again by the phase step of an accepted frame
    }
  }
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_l2_stats(const __grid_constant__ L2Batch b) {
  grid_dep_launch();
  l2_stage_stats<N>(b, blockIdx.y, blockIdx.x);
}

// combine the row-block partials in rank order (identical in every block); called by one warp:
// its lanes fetch the B records in parallel into `rec`, lane 0 combines them
template <int N>
__device__ void l2_combine(const L2Stream& S, const KParams& P, float* g, float (*rec)[8], int lane) {
  constexpr int B = N / kT;
  for (int k = lane; k < B; k += 32)
#pragma unroll
    for (int j = 0; j < 7; ++j) rec[k][j] = S.part[8 * k + j];
  __syncwarp();
  if (lane != 0) return;
  const float nb = static_cast<float>(kT * N);
  float n_a = nb, q_a = rec[0][2];
  float2 m_a = make_float2(rec[0][0], rec[0][1]);
  float t0 = rec[0][3], t1 = rec[0][4], t2 = rec[0][5], t3 = rec[0][6];
  for (int k = 1; k < B; ++k) {
    const float* o = rec[k];
    const float nn = n_a + nb;
    const float2 d = make_float2(o[0] - m_a.x, o[1] - m_a.y);
    const float f = nb / nn;
    m_a = make_float2(fmaf(d.x, f, m_a.x), fmaf(d.y, f, m_a.y));
    q_a = q_a + o[2] + c_abs2(d) * (n_a * f);
    n_a = nn;
    t0 += o[3]; t1 += o[4]; t2 += o[5]; t3 += o[6];
  }
  const float scale = sqrtf(static_cast<float>(N) * static_cast<float>(N) / q_a);
  const bool finite = isfinite(m_a.x) && isfinite(m_a.y) && isfinite(q_a) && q_a > 0.f && isfinite(scale);
  g[0] = m_a.x;
  g[1] = m_a.y;
  g[2] = scale;
  g[3] = (P.tilt_mode && t1 > 0.f) ? t0 / t1 : 0.f;
  g[4] = (P.tilt_mode && t3 > 0.f) ? t2 / t3 : 0.f;
  g[5] = finite ? 0.f : 1.f;
}

// ---- s2: prologue and row IFFT of the pupil rows; transposed store into fb ------------------
template <int N, int V>
__device__ __forceinline__ void l2_stage_rows_inv(const L2Batch& b, const float2* twg, int sid, int bx, int first, unsigned char* smem) {
  const L2Stream& S = b.st[sid];
  const KParams& P = b.prm[sid];
  const float2* y = b.ytab != nullptr ? b.ytab[b.ytab_base + sid] : S.y;
  float2* tw = reinterpret_cast<float2*>(smem);
  // row tile with stride N + 4: the transposed accesses (8 rows x 4 columns per warp) hit
  // 16 bank pairs
  constexpr int RW = N + 4;
  float2* rows = tw + N;  // kTr rows x RW
  __shared__ float g[8];
  __shared__ float rec[N / kT][8];
  for (int i = threadIdx.x; i < N; i += kRowThreads) tw[i] = twg[i];
  grid_dep_wait();
  if (first && threadIdx.x < 32) l2_combine<N>(S, P, g, rec, threadIdx.x);
  if (threadIdx.x == 0) {
    if (first) {
      if (bx == 0) {
        float* st = S.part + 8 * (N / kT);  // combined statistics for the later stages
        for (int k = 0; k < 6; ++k) st[k] = g[k];
        if (g[5] != 0.f) {
          *S.flag = 1;
          if (S.status != nullptr) atomicOr(S.status, kStatusNonFinite);
        }
      }
    } else {
      const float* st = S.part + 8 * (N / kT);
      for (int k = 0; k < 6; ++k) g[k] = st[k];
    }
  }
  __syncthreads();
  if (g[5] != 0.f) return;
  const float2 ymean = make_float2(g[0], g[1]);
  const float scale = g[2], tx = g[3], ty = g[4];
  const float cc = 0.5f * static_cast<float>(N - 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rho = kTr * bx + warp;
  const int dy2 = ap_dist2(rho, N);
  float2* rb = rows + warp * RW;
  float* pr = S.phi + static_cast<size_t>(rho) * N;
  if (dy2 <= P.ap_lim) {
    const float tyr = ty * (static_cast<float>(rho) - cc);
    constexpr int PER = N / 32;
    float pv[PER];
    float2 yv[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {  // every load before the first store
      const int x = lane + 32 * j;
      const bool in = ap_dist2(x, N) + dy2 <= P.ap_lim;
      pv[j] = in ? pr[x] : 0.f;
      yv[j] = in ? y[static_cast<size_t>(rho) * N + x] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int x = lane + 32 * j;
      float2 u = make_float2(0.f, 0.f);
      float ph = 0.f;
      if (ap_dist2(x, N) + dy2 <= P.ap_lim) {
        ph = pv[j];
        if (first && P.tilt_mode) ph = wrap_pi(ph - fmaf(tx, static_cast<float>(x) - cc, tyr));
        const float2 yt = c_scale(c_sub(yv[j], ymean), scale);
        float sn, cs;
        sincosf(ph, &sn, &cs);
        u = make_float2(fmaf(yt.x, cs, yt.y * sn), fmaf(yt.y, cs, -yt.x * sn));
      }
      pr[x] = ph;  // the state keeps phi' (tip/tilt removed) until the phase step
      rb[swz(x)] = u;
    }
    __syncwarp();
    fft_row<N, +1, V>(rb, tw, lane);
  } else {
    for (int x = lane; x < N; x += 32) {
      rb[swz(x)] = make_float2(0.f, 0.f);
      pr[x] = 0.f;
    }
  }
  __syncthreads();
  // fb is column-major: fb[x N + rho]; 8 threads write the 8 rows of one column.  Rows outside
  // the aperture are zero and are not stored: the column pass fills them in itself.
  for (int i = threadIdx.x; i < kTr * N; i += kRowThreads) {
    const int x = i / kTr, r = i - x * kTr;
    if (ap_dist2(kTr * bx + r, N) <= P.ap_lim)
      S.fb[static_cast<size_t>(x) * N + kTr * bx + r] = rows[r * RW + swz(x)];
  }
}

template <int N, int V>
__global__ void __launch_bounds__(kRowThreads) k_l2_rows_inv(const __grid_constant__ L2Batch b, int first) {
  extern __shared__ __align__(128) unsigned char smem[];
  grid_dep_launch();
  l2_stage_rows_inv<N, V>(b, b.tw, blockIdx.y, blockIdx.x, first, smem);
}

// ---- s3: column IFFT, r-init + E-step, column FFT of mu; transposed store into fa ----------
// AUX: the stream has the post-step M-steps' side buffer (the instantiation without it is the
// plain stage; a kernel picks one per stream, uniformly over each block)
template <int N, int V, bool AUX>
__device__ __forceinline__ void l2_stage_cols(const L2Batch& b, const float2* twg, int sid, int bx, int first, int last,
                                              unsigned char* smem) {
  const L2Stream& S = b.st[sid];
  const KParams& P = b.prm[sid];
  grid_dep_wait();
  if (frame_dropped(S)) return;
  // sigma^2 of this frame: the stream's running estimate when it is re-estimated (written by the
  // previous frame's post kernel), else the parameter
  float* aux = AUX ? b.aux[sid] : nullptr;
  const float nv = AUX ? aux[0] : P.noise_var;
  const bool aux_out = AUX && last;  // side outputs of the frame's last iteration
  float2* tw = reinterpret_cast<float2*>(smem);
  // column tiles with stride N + 4: the transposed accesses (8 columns x 4 rows per warp) hit
  // 32 distinct banks (16 bank pairs for the complex tile)
  constexpr int CW = N + 4;
  float2* cols = tw + N;                                    // kTc columns x CW
  float* rt = reinterpret_cast<float*>(cols + kTc * CW);    // kTc x CW: r, then r-init
  float* stile = rt + kTc * CW;                             // kTc x CW: s
  for (int i = threadIdx.x; i < N; i += kColThreads) tw[i] = twg[i];
  const int x0 = kTc * bx;
  {
    // every load of a thread is issued before its first store (the shared-memory stores could
    // alias the loads' generic addresses otherwise, which would serialise them)
    constexpr int PER = kTc * N / kColThreads;
    float2 fv[PER];
    float rv[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = threadIdx.x + kColThreads * j, c = i / N, rho = i - c * N;
      fv[j] = ap_dist2(rho, N) <= P.ap_lim ? S.fb[static_cast<size_t>(x0 + c) * N + rho] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {  // coalesced 32-byte row segments
      const int i = threadIdx.x + kColThreads * j, rho = i / kTc, c = i - rho * kTc;
      rv[j] = S.r[static_cast<size_t>(rho) * N + x0 + c];
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = threadIdx.x + kColThreads * j, c = i / N, rho = i - c * N;
      cols[c * CW + swz(rho)] = fv[j];
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = threadIdx.x + kColThreads * j, rho = i / kTc, c = i - rho * kTc;
      rt[c * CW + rho] = rv[j];
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* cb = cols + warp * CW;
  float* rc = rt + warp * CW;
  float* sc = stile + warp * CW;
  fft_row<N, +1, V>(cb, tw, lane);
  const float invN = 1.f / static_cast<float>(N);
  float csum = 0.f;  // sum of the posterior variances C = sigma^2 w (side output)
  for (int rho = lane; rho < N; rho += 32) {
    const float2 bb = c_scale(cb[swz(rho)], invN);
    const float rp = rc[rho];
    const float ri = first ? fmaxf(fmaf(P.lam1, rp, P.lam_alpha * c_abs2(bb)), P.r_floor) : rp;
    const float w = ri / (ri + nv);
    const float2 mu = c_scale(bb, w);
    cb[swz(rho)] = mu;
    rc[rho] = ri;
    sc[rho] = fmaf(nv, w, c_abs2(mu));
    if constexpr (AUX) csum += nv * w;
  }
  __shared__ float cred[kTc];
  if constexpr (AUX) {
    if (aux_out) {
      csum = warp_sum(csum);
      if (lane == 0) cred[warp] = csum;
    }
  }
  __syncwarp();
  fft_row<N, -1, V>(cb, tw, lane);
  __syncthreads();
  if constexpr (AUX) {
    if (aux_out && threadIdx.x == 0) {  // this block's sum, its columns in order
      float sc0 = 0.f;
      for (int w2 = 0; w2 < kTc; ++w2) sc0 += cred[w2];
      aux[kAuxPart + 2 * bx + 1] = sc0;
    }
  }
  for (int i = threadIdx.x; i < kTc * N; i += kColThreads) {
    const int rho = i / kTc, c = i - rho * kTc;
    const size_t gi = static_cast<size_t>(rho) * N + x0 + c;
    const float ri = rt[c * CW + rho];
    S.r0[gi] = ri;
    S.r[gi] = ri;  // the ICD sweep starts from r-init
    S.s[gi] = stile[c * CW + rho];
    if (ap_dist2(rho, N) <= P.ap_lim) S.fa[gi] = cols[c * CW + swz(rho)];
  }
}

template <int N, int V>
__global__ void __launch_bounds__(kColThreads) k_l2_cols(const __grid_constant__ L2Batch b, int first, int last) {
  extern __shared__ __align__(128) unsigned char smem[];
  grid_dep_launch();
  l2_stage_cols<N, V, false>(b, b.tw, blockIdx.y, blockIdx.x, first, last, smem);
}

// the same stage for a launch whose streams all have the post-step side buffer (a separate
// kernel, so that the plain one keeps its own register allocation)
template <int N, int V>
__global__ void __launch_bounds__(kColThreads) k_l2_cols_aux(const __grid_constant__ L2Batch b, int first, int last) {
  extern __shared__ __align__(128) unsigned char smem[];
  grid_dep_launch();
  l2_stage_cols<N, V, true>(b, b.tw, blockIdx.y, blockIdx.x, first, last, smem);
}

// ---- s4: row FFT of mu and phase M-step ------------------------------------------------------
template <int N, int V, bool AUX>
__device__ __forceinline__ void l2_stage_rows_fwd(const L2Batch& b, const float2* twg, int sid, int bx, int last,
                                                  unsigned char* smem) {
  const L2Stream& S = b.st[sid];
  const KParams& P = b.prm[sid];
  grid_dep_wait();
  if (frame_dropped(S)) return;
  const float2* y = b.ytab != nullptr ? b.ytab[b.ytab_base + sid] : S.y;
  float2* tw = reinterpret_cast<float2*>(smem);
  // row tile with stride N + 4: the transposed accesses (8 rows x 4 columns per warp) hit
  // 16 bank pairs
  constexpr int RW = N + 4;
  float2* rows = tw + N;  // kTr rows x RW
  float* ev = reinterpret_cast<float*>(rows + kTr * RW);  // kTr rows x N: a (|y~|^2 + |z|^2)
  float* aux = AUX ? b.aux[sid] : nullptr;
  const bool aux_out = AUX && last;                       // side outputs of the frame's last iteration
  for (int i = threadIdx.x; i < N; i += kRowThreads) tw[i] = twg[i];
  const float* st = S.part + 8 * (N / kT);
  const float2 ymean = make_float2(st[0], st[1]);
  const float scale = st[2];
  const int gs = P.g_shift, G = 1 << gs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rho = kTr * bx + warp;
  const int dy2 = ap_dist2(rho, N);
  const bool row_ap = dy2 <= P.ap_lim;
  float2* rb = rows + warp * RW;
  constexpr int PER = N / 32;
  if (row_ap) {
    float2 fv[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) fv[j] = S.fa[static_cast<size_t>(rho) * N + lane + 32 * j];
#pragma unroll
    for (int j = 0; j < PER; ++j) rb[swz(lane + 32 * j)] = fv[j];
  }
  __syncthreads();
  if (row_ap) fft_row<N, -1, V>(rb, tw, lane);
  const float invN = 1.f / static_cast<float>(N);
  float2 yv[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int x = lane + 32 * j;
    yv[j] = row_ap && ap_dist2(x, N) + dy2 <= P.ap_lim ? y[static_cast<size_t>(rho) * N + x] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int x = lane + 32 * j;
    float2 v = make_float2(0.f, 0.f);
    float e = 0.f;
    if (row_ap && ap_dist2(x, N) + dy2 <= P.ap_lim) {
      const float2 z = c_scale(rb[swz(x)], invN);
      const float2 yt = c_scale(c_sub(yv[j], ymean), scale);
      v = make_float2(fmaf(yt.x, z.x, yt.y * z.y), fmaf(yt.y, z.x, -yt.x * z.y));
      if constexpr (AUX) e = aux_out ? c_abs2(yt) + c_abs2(z) : 0.f;
    }
    for (int o = 1; o < G; o <<= 1) {  // sum over the G consecutive x of the tile
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      if constexpr (AUX) e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    rb[swz(x)] = v;
    if constexpr (AUX) ev[warp * N + x] = e;
  }
  __syncthreads();
  const int l0 = warp & ~(G - 1);
  float* pr = S.phi + static_cast<size_t>(rho) * N;
  for (int x = lane; x < N; x += 32) {
    if (row_ap && ap_dist2(x, N) + dy2 <= P.ap_lim) {
      float2 v = rows[l0 * RW + swz(x)];
      for (int j = 1; j < G; ++j) v = c_add(v, rows[(l0 + j) * RW + swz(x)]);
      if (v.x != 0.f || v.y != 0.f) pr[x] = atan2f(v.y, v.x);  // else phi' is kept
    }
  }
  if (AUX && aux_out) {
    // Side outputs for the post kernel, per G x G tile of this block's rows: the tile sums v_t
    // and E_t.  With the phase prior they go to the tile grid; otherwise the tile phase is
    // angle(v_t) and the pupil residual |y~ - e^{j phi} z|^2 over the tile is E_t - 2 |v_t|,
    // summed here.  Then this block's residual, its warps in order.
    const int NT = N >> gs;
    float res = 0.f;
    for (int t = threadIdx.x; t < (kTr >> gs) * NT; t += kRowThreads) {
      const int tl = t / NT, tx = t - tl * NT;
      const int lt = tl << gs, xt = tx << gs;
      float2 v = rows[lt * RW + swz(xt)];
      float e = ev[lt * N + xt];
      for (int j = 1; j < G; ++j) {
        v = c_add(v, rows[(lt + j) * RW + swz(xt)]);
        e += ev[(lt + j) * N + xt];
      }
      if (b.aux_tiles[sid]) {
        const int T = (kTr * bx + lt) >> gs;
        if (tile_in_pupil(T, tx, gs, N, P.ap_lim))
          reinterpret_cast<float4*>(aux + kAuxTiles)[T * NT + tx] = make_float4(v.x, v.y, e, 0.f);
      } else {
        res += e - 2.f * sqrtf(fmaf(v.x, v.x, v.y * v.y));
      }
    }
    __shared__ float rred[kTr];
    res = warp_sum(res);
    if (lane == 0) rred[warp] = res;
    __syncthreads();
    if (threadIdx.x == 0) {
      float sr = 0.f;
      for (int w2 = 0; w2 < kTr; ++w2) sr += rred[w2];
      aux[kAuxPart + 2 * bx] = sr;
      if (bx == 0) aux[1] = 1.f;  // the frame was accepted
    }
  }
}

template <int N, int V>
__global__ void __launch_bounds__(kRowThreads) k_l2_rows_fwd(const __grid_constant__ L2Batch b, int last) {
  extern __shared__ __align__(128) unsigned char smem[];
  grid_dep_launch();
  l2_stage_rows_fwd<N, V, false>(b, b.tw, blockIdx.y, blockIdx.x, last, smem);
}

// with the post-step side outputs (four blocks per SM at 512^2 keep it at 64 registers)
template <int N, int V>
__global__ void __launch_bounds__(kRowThreads, N == 512 ? 4 : 6) k_l2_rows_fwd_aux(const __grid_constant__ L2Batch b,
                                                                                  int last) {
  extern __shared__ __align__(128) unsigned char smem[];
  grid_dep_launch();
  l2_stage_rows_fwd<N, V, true>(b, b.tw, blockIdx.y, blockIdx.x, last, smem);
}

// ---- s5: surrogate pair weights at the sweep's entry values ---------------------------------
template <int N>
__device__ __forceinline__ void l2_stage_weights(const L2Batch& b, int sid, int bx) {
  const L2Stream& S = b.st[sid];
  const KParams& P = b.prm[sid];
  grid_dep_wait();
  if (frame_dropped(S)) return;
  constexpr int M = N * N;
  auto wgt = [&](float d) { return prior_weight_fast(d, P.w0, P.inv_tsig, P.q_minus_p, P.q_over_p); };
  // kWPx pixels per thread (the grid covers the image once); all their loads are issued
  // before the first store, which could alias them otherwise
  constexpr int kWPx = 2;
  const int i0 = bx * blockDim.x * kWPx + threadIdx.x;
  float a[kWPx], vE[kWPx], vS[kWPx], vSE[kWPx], vSW[kWPx];
#pragma unroll
  for (int u = 0; u < kWPx; ++u) {
    const int i = i0 + u * blockDim.x, rho = i / N, x = i - rho * N;
    const bool rt = x + 1 < N, dn = rho + 1 < N, lf = x > 0;
    a[u] = S.r0[i];
    vE[u] = rt ? S.r0[i + 1] : 0.f;
    vS[u] = dn ? S.r0[i + N] : 0.f;
    vSE[u] = (rt && dn) ? S.r0[i + N + 1] : 0.f;
    vSW[u] = (lf && dn) ? S.r0[i + N - 1] : 0.f;
  }
#pragma unroll
  for (int u = 0; u < kWPx; ++u) {
    const int i = i0 + u * blockDim.x, rho = i / N, x = i - rho * N;
    const bool rt = x + 1 < N, dn = rho + 1 < N, lf = x > 0;
    S.beta[i] = rt ? kBnn * wgt(a[u] - vE[u]) : 0.f;
    S.beta[M + i] = dn ? kBnn * wgt(a[u] - vS[u]) : 0.f;
    S.beta[2 * M + i] = (rt && dn) ? kBdiag * wgt(a[u] - vSE[u]) : 0.f;
    S.beta[3 * M + i] = (lf && dn) ? kBdiag * wgt(a[u] - vSW[u]) : 0.f;
  }
}

template <int N>
__global__ void __launch_bounds__(256) k_l2_weights(const __grid_constant__ L2Batch b) {
  grid_dep_launch();
  l2_stage_weights<N>(b, blockIdx.y, blockIdx.x);
}

// ---- s6: one ICD colour ---------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void l2_stage_colour(const L2Batch& b, int sid, int bx, int c, int nbx) {
  const L2Stream& S = b.st[sid];
  const KParams& P = b.prm[sid];
  grid_dep_wait();
  if (frame_dropped(S)) return;
  constexpr int M = N * N;
  const int cx = c & 1, cy = c >> 1;
  for (int k = bx * blockDim.x + threadIdx.x; k < M / 4; k += nbx * blockDim.x) {
    const int rho = cy + 2 * (k / (N / 2)), x = cx + 2 * (k % (N / 2));
    const int i = rho * N + x;
    const bool up = rho > 0, dn = rho + 1 < N, lf = x > 0, rt = x + 1 < N;
    const float* bE = S.beta;
    const float* bS = S.beta + M;
    const float* bSE = S.beta + 2 * M;
    const float* bSW = S.beta + 3 * M;
    const float* r = S.r;
    const float wE = bE[i], wS = bS[i], wSE = bSE[i], wSW = bSW[i];
    const float wW = lf ? bE[i - 1] : 0.f;
    const float wN = up ? bS[i - N] : 0.f;
    const float wNW = (up && lf) ? bSE[i - N - 1] : 0.f;
    const float wNE = (up && rt) ? bSW[i - N + 1] : 0.f;
    const float rW = lf ? r[i - 1] : 0.f, rE = rt ? r[i + 1] : 0.f;
    const float rN = up ? r[i - N] : 0.f, rSo = dn ? r[i + N] : 0.f;
    const float rNW = (up && lf) ? r[i - N - 1] : 0.f, rNE = (up && rt) ? r[i - N + 1] : 0.f;
    const float rSW = (dn && lf) ? r[i + N - 1] : 0.f, rSE = (dn && rt) ? r[i + N + 1] : 0.f;
    const float Wsum = ((wN + wS) + (wW + wE)) + ((wNW + wNE) + (wSW + wSE));
    float Csum = wN * rN;
    Csum = fmaf(wS, rSo, Csum);
    Csum = fmaf(wW, rW, Csum);
    Csum = fmaf(wE, rE, Csum);
    Csum = fmaf(wNW, rNW, Csum);
    Csum = fmaf(wNE, rNE, Csum);
    Csum = fmaf(wSW, rSW, Csum);
    Csum = fmaf(wSE, rSE, Csum);
    S.r[i] = fmaxf(icd_root_from(Wsum, Csum, S.s[i], S.r0[i]), P.r_floor);
  }
}

template <int N>
__global__ void __launch_bounds__(256) k_l2_colour(const __grid_constant__ L2Batch b, int c) {
  grid_dep_launch();
  l2_stage_colour<N>(b, blockIdx.y, blockIdx.x, c, gridDim.x);
}

template <int N>
constexpr size_t rows_smem() { return sizeof(float2) * (N + kTr * (N + 4)); }
template <int N>
constexpr size_t rows_smem_aux() { return rows_smem<N>() + sizeof(float) * kTr * N; }  // + the E rows
template <int N>
constexpr size_t cols_smem() { return sizeof(float2) * (N + kTc * (N + 4)) + 2 * sizeof(float) * kTc * (N + 4); }

// launch with programmatic stream serialization (the kernel waits for its predecessor itself)
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// every stream of `b` has the post-step side buffer, or none (the caller forms such launches)
template <int N, int V>
cudaError_t l2_step(const L2Batch& b, int n_k, cudaStream_t st) {
  const bool aux = b.aux[0] != nullptr;
  const dim3 grid(N / kT, b.count), blk(kThreads);
  const dim3 rgrid(N / kTr, b.count), rblk(kRowThreads);
  const dim3 cgrid2(N / kTc, b.count), cblk(kColThreads);
  // pixel kernels: two pixels per thread for the weights, one per thread for a colour
  const dim3 wgrid(N * N / (2 * 256), b.count), cgrid(N * N / (4 * 256), b.count);
  cudaError_t e = launch_pdl(k_l2_stats<N>, grid, blk, 0, st, b);
  for (int it = 0; it < n_k && e == cudaSuccess; ++it) {
    const int first = it == 0 ? 1 : 0;
    e = launch_pdl(k_l2_rows_inv<N, V>, rgrid, rblk, rows_smem<N>(), st, b, first);
    const int last = it == n_k - 1 ? 1 : 0;
    if (e == cudaSuccess)
      e = launch_pdl(aux ? k_l2_cols_aux<N, V> : k_l2_cols<N, V>, cgrid2, cblk, cols_smem<N>(), st, b, first, last);
    if (e == cudaSuccess)
      e = launch_pdl(aux ? k_l2_rows_fwd_aux<N, V> : k_l2_rows_fwd<N, V>, rgrid, rblk,
                     aux ? rows_smem_aux<N>() : rows_smem<N>(), st, b, last);
    if (e == cudaSuccess) e = launch_pdl(k_l2_weights<N>, wgrid, dim3(256), 0, st, b);
    for (int c = 0; c < 4 && e == cudaSuccess; ++c) e = launch_pdl(k_l2_colour<N>, cgrid, dim3(256), 0, st, b, c);
  }
  return e;
}

template <int N, int V>
cudaError_t l2_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_l2_rows_inv<N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(rows_smem<N>()));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_l2_cols<N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(cols_smem<N>()));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_l2_rows_fwd<N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(rows_smem<N>()));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_l2_cols_aux<N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(cols_smem<N>()));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_l2_rows_fwd_aux<N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(rows_smem_aux<N>()));
  return e;
}

// ---- one persistent launch per batched step -----------------------------------------------
// The nine stages of every stream of the batch (any mix of the staged grid sizes) in one
// cooperative launch: at each stage the grid's blocks take the stage's work items -- (stream,
// block) pairs of the chained kernels, listed group by group -- in a block-strided loop, and a
// grid-wide barrier separates the stages.  Every item runs the same stage function as the
// chained kernels (256 threads), so the results are bit for bit those of the chained launches.
constexpr int kPersistThreads = 256;
constexpr uint64_t kBarrierLimitNs = 200000000ull;  // 200 ms; a stage takes tens of microseconds

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Items (blocks of the chained kernel) of stage `stage` for one stream of grid n: 0 statistics,
// 1 prologue + row IFFT, 2 column pass, 3 row FFT + phase step, 4 pair weights, 5-8 colours.
__device__ __forceinline__ int stage_items(int stage, int n) {
  switch (stage) {
    case 0: return n / kT;
    case 1: case 3: return n / kTr;
    case 2: return n / kTc;
    case 4: return n * n / 512;
    default: return n * n / 1024;
  }
}

// Each stage of each grid size is its own (not inlined) function, so that the persistent
// kernel's register budget is that of its largest stage rather than of all of them inlined
// together.
template <int N>
__device__ __noinline__ void pi_stats(const L2Batch& b, int sid, int bx) { l2_stage_stats<N>(b, sid, bx); }
template <int N>
__device__ __noinline__ void pi_rows_inv(const L2Batch& b, const float2* tw, int sid, int bx, int first,
                                         unsigned char* smem) {
  l2_stage_rows_inv<N, 0>(b, tw, sid, bx, first, smem);
}
template <int N>
__device__ __noinline__ void pi_cols(const L2Batch& b, const float2* tw, int sid, int bx, int first, int last,
                                     unsigned char* smem) {
  l2_stage_cols<N, 0, false>(b, tw, sid, bx, first, last, smem);  // no side buffers here
}
template <int N>
__device__ __noinline__ void pi_rows_fwd(const L2Batch& b, const float2* tw, int sid, int bx, int last,
                                         unsigned char* smem) {
  l2_stage_rows_fwd<N, 0, false>(b, tw, sid, bx, last, smem);
}
template <int N>
__device__ __noinline__ void pi_weights(const L2Batch& b, int sid, int bx) { l2_stage_weights<N>(b, sid, bx); }
template <int N>
__device__ __noinline__ void pi_colour(const L2Batch& b, int sid, int bx, int c) {
  l2_stage_colour<N>(b, sid, bx, c, N * N / 1024);
}

template <int N>
__device__ __forceinline__ void persist_item(const L2Batch& b, const float2* tw, int stage, int first, int last,
                                             int sid, int bx, unsigned char* smem) {
  switch (stage) {
    case 0: pi_stats<N>(b, sid, bx); break;
    case 1: pi_rows_inv<N>(b, tw, sid, bx, first, smem); break;
    case 2: pi_cols<N>(b, tw, sid, bx, first, last, smem); break;
    case 3: pi_rows_fwd<N>(b, tw, sid, bx, last, smem); break;
    case 4: pi_weights<N>(b, sid, bx); break;
    default: pi_colour<N>(b, sid, bx, stage - 5); break;
  }
}

// Grid-wide barrier: thread 0 of each block publishes the block's writes (fence), arrives on
// bar[0] and waits for the last arrival to advance the generation bar[1]; the wait polls with
// a device-time limit, after which it raises the abort word bar[2].  Returns false (to every
// thread of the block) when the barrier was abandoned, by this block or another.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* vabort = bar + 2;
    int res = 1;
    const unsigned gen = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*vgen == gen) {
        if (*vabort != 0u) { res = 0; break; }
        if (global_ns() - t0 > kBarrierLimitNs) {
          atomicExch(bar + 2, 1u);
          res = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = res;
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(kPersistThreads, 4) k_l2_persistent(const __grid_constant__ L2Persist p) {
  extern __shared__ __align__(128) unsigned char smem[];
  grid_dep_wait();
  for (int it = 0; it < p.n_k; ++it) {
    const int first = it == 0 ? 1 : 0, last = it == p.n_k - 1 ? 1 : 0;
    for (int stage = it == 0 ? 0 : 1; stage < 9; ++stage) {
      int total = 0;
      for (int g = 0; g < p.groups; ++g) total += p.count[g] * stage_items(stage, p.n[g]);
      for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int g = 0, local = item;
        for (; g < p.groups - 1; ++g) {
          const int ng = p.count[g] * stage_items(stage, p.n[g]);
          if (local < ng) break;
          local -= ng;
        }
        const int per = stage_items(stage, p.n[g]);
        const int sid = p.first[g] + local / per, bx = local % per;
        switch (p.n[g]) {
          case 512: persist_item<512>(p.b, p.tw[g], stage, first, last, sid, bx, smem); break;
          case 256: persist_item<256>(p.b, p.tw[g], stage, first, last, sid, bx, smem); break;
          default: persist_item<128>(p.b, p.tw[g], stage, first, last, sid, bx, smem); break;
        }
        __syncthreads();  // the item's shared scratch is free for the next item
      }
      if (it == p.n_k - 1 && stage == 8) break;  // no barrier after the last stage
      if (!grid_barrier(p.bar, gridDim.x)) {
        // abandoned: every stream of the launch reports the expired wait; its state is left
        // part-way through the step (reload a checkpoint)
        if (threadIdx.x == 0 && blockIdx.x == 0)
          for (int i = 0; i < p.b.count; ++i)
            if (p.b.st[i].status != nullptr) atomicOr(p.b.st[i].status, kStatusTimeout);
        return;
      }
    }
  }
}

}  // namespace

cudaError_t launch_step_l2_persistent(const L2Persist& p, cudaStream_t st) {
  // shared memory of the largest stage of the largest grid in the launch
  int nmax = 0;
  for (int g = 0; g < p.groups; ++g) nmax = p.n[g] > nmax ? p.n[g] : nmax;
  const size_t smem = nmax == 512 ? cols_smem<512>() : nmax == 256 ? cols_smem<256>() : cols_smem<128>();
  static thread_local int dev_cached = -1;
  static thread_local int blocks_cached[3] = {0, 0, 0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int slot = nmax == 512 ? 0 : nmax == 256 ? 1 : 2;
  if (dev != dev_cached) {
    blocks_cached[0] = blocks_cached[1] = blocks_cached[2] = 0;
    dev_cached = dev;
  }
  if (blocks_cached[slot] == 0) {
    e = cudaFuncSetAttribute(k_l2_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(cols_smem<512>()));
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_l2_persistent, kPersistThreads, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    blocks_cached[slot] = per_sm * sms;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks_cached[slot]);
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_l2_persistent, p);
}

size_t l2_scratch_bytes(int n) {
  if (n != 128 && n != 256 && n != 512) return 0;
  const size_t M = static_cast<size_t>(n) * n;
  // fa, fb (complex), r-init, s, 4 weight images, row-block partials + combined stats, flag
  return 2 * M * sizeof(float2) + 6 * M * sizeof(float) + (8 * (n / kT) + 16) * sizeof(float) + 256;
}

L2Stream l2_stream_view(void* scratch, int n) {
  const size_t M = static_cast<size_t>(n) * n;
  char* p = static_cast<char*>(scratch);
  L2Stream s{};
  s.fa = reinterpret_cast<float2*>(p);
  s.fb = s.fa + M;
  s.r0 = reinterpret_cast<float*>(s.fb + M);
  s.s = s.r0 + M;
  s.beta = s.s + M;
  s.part = s.beta + 4 * M;
  s.flag = reinterpret_cast<int*>(s.part + 8 * (n / kT) + 16);
  s.bar = reinterpret_cast<unsigned*>(s.flag + 4);  // inside the 256-byte tail
  return s;
}

cudaError_t configure_l2(int n) {
  switch (n) {
    case 128: return l2_configure<128, 0>();
    case 256: return l2_configure<256, 0>();
    case 512: return l2_configure<512, 0>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step_l2(int n, int schedule, const L2Batch& b, int n_k, cudaStream_t st) {
  (void)schedule;  // the staged kernels use one radix schedule per grid size
  switch (n) {
    case 128: return l2_step<128, 0>(b, n_k, st);
    case 256: return l2_step<256, 0>(b, n_k, st);
    case 512: return l2_step<512, 0>(b, n_k, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ddh
