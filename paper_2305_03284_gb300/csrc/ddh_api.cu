// C ABI of libddh (declarations and contracts in include/ddh.h).
//
// Host side only: argument validation, device state ownership, parameter derivation, the
// per-device twiddle tables and kernel attributes, error latching.  Every compute step is one
// of the kernels in ddh_step.cu.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ddh.h"
#include "ddh_internal.h"
#include "ddh_eval.cuh"
#include "ddh_kernels.cuh"

namespace ddh {
cudaError_t launch_wait_selftest(unsigned* status, uint64_t limit_ns, cudaStream_t st);  // ddh_selftest.cu
}  // namespace ddh

struct ddh_state {
  ddh_params prm;
  ddh::KParams kp;
  cudaStream_t stream;
  int device;
  float* r;
  float* phi;
  unsigned* status;
  float2* ystage;
  float* scalar;
  bool staged;      // steps run on the L2-staged kernels (exec_path), else the cluster kernel
  void* l2scratch;  // working images of the L2-staged kernels (staged states only)
  const float2* tw;
  int64_t frame;
  int64_t ap_count;
  // side buffer of the tile-phase prior and sigma^2 M-steps (ddh::aux_floats floats; null
  // while neither is enabled): sigma^2 in use, the step's partial sums and tile sums
  float* aux = nullptr;
  // pipelined host-buffer steps (ddh_step_host_async), set up on first use: two device staging
  // slots (ystage and hstage2) filled on a copy-in stream, events that order a slot's copy
  // before its step and the step before the slot's next copy, and a ring of completion events
  cudaStream_t cin = nullptr;
  float2* hstage2 = nullptr;
  cudaEvent_t ev_in[2] = {};
  cudaEvent_t ev_used[2] = {};
  cudaEvent_t ev_done[8] = {};
  int64_t hcount = 0;
};

namespace {

constexpr int kVersion = 101;
constexpr int kMaxDevices = 64;
thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DDH_ENOMEM : DDH_ECUDA;
}
#define DDH_CUDA(call)                         \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)
// `dev` current until the enclosing scope ends (the caller's device is restored then)
#define DDH_ON_DEVICE(dev)                 \
  DdhDeviceGuard ddh_dev_guard_(dev);      \
  DDH_CUDA(ddh_dev_guard_.error())

bool supported_n(int n) { return n == 32 || n == 64 || n == 128 || n == 256 || n == 512; }
bool cluster_n(int n) { return n != 512; }  // grids the cluster kernel (and k_strehl, k_fft2) handles
bool staged_n(int n) { return n == 128 || n == 256 || n == 512; }  // grids of the L2-staged kernels
int n_slot(int n) { return n == 32 ? 3 : n == 64 ? 0 : n == 128 ? 1 : n == 256 ? 2 : 4; }
// the kernels a state with parameters `p` steps on (exec_path resolved)
bool staged_path(const ddh_params& p) {
  return p.exec_path == DDH_PATH_STAGED || (p.exec_path == DDH_PATH_DEFAULT && !cluster_n(p.n));
}

std::mutex g_mu;
bool g_configured[kMaxDevices][5] = {};     // cluster kernels (N <= 256) and the twiddle table
bool g_configured_l2[kMaxDevices][5] = {};  // L2-staged kernels
float2* g_twiddle[kMaxDevices][5] = {};
int g_schedule[kMaxDevices][5] = {};  // FFT radix schedule used for each grid size
// streams per launch chunk of the L2-staged kernels, per grid size (0: the default, 16)
int g_chunk[kMaxDevices][5] = {};
// 1: a batch's staged streams run as one persistent launch per step (ddh_set_staged_persistent)
int g_persistent[kMaxDevices] = {};
int staged_chunk(int dev, int n) {
  const int c = g_chunk[dev][n_slot(n)];
  return c > 0 ? c : 16;
}

// Library-owned side streams that let the grid-size groups of one batch run concurrently.
constexpr int kGroups = 7;  // (grid, path) groups of a batch: 4 cluster sizes, 3 staged sizes
struct SideStreams {
  bool ready = false;
  cudaStream_t s[kGroups] = {};
  cudaEvent_t fork = nullptr, join[kGroups] = {};
};
SideStreams g_side[kMaxDevices];

int side_streams(int dev, SideStreams** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  SideStreams& ss = g_side[dev];
  if (!ss.ready) {
    for (int i = 0; i < kGroups; ++i) {
      DDH_CUDA(cudaStreamCreateWithFlags(&ss.s[i], cudaStreamNonBlocking));
      DDH_CUDA(cudaEventCreateWithFlags(&ss.join[i], cudaEventDisableTiming));
    }
    DDH_CUDA(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
    ss.ready = true;
  }
  *out = &ss;
  return DDH_OK;
}

// Per-device, per-N setup: kernel attributes and the twiddle table exp(-2 pi i t / N),
// evaluated in double precision and rounded once to float; `staged`: also the L2-staged
// kernels' attributes.
int device_setup(int dev, int n, const float2** tw, bool staged = false) {
  if (dev < 0 || dev >= kMaxDevices) return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  const int s = n_slot(n);
  if (staged && !g_configured_l2[dev][s]) {
    DDH_CUDA(ddh::configure_l2(n));
    g_configured_l2[dev][s] = true;
  }
  if (!g_configured[dev][s]) {
    int active = 1;
    if (cluster_n(n)) DDH_CUDA(ddh::configure(n, &active));
    if (active < 1) {
      std::snprintf(g_cuda_err, sizeof(g_cuda_err), "no resident cluster of %d CTAs x %zu B shared memory", n / 16,
                    ddh::step_smem_bytes(n));
      return DDH_ECUDA;
    }
    std::vector<float2> h(n);
    for (int t = 0; t < n; ++t) {
      const double a = -2.0 * M_PI * static_cast<double>(t) / static_cast<double>(n);
      h[t] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
    }
    float2* d = nullptr;
    DDH_CUDA(cudaMalloc(&d, sizeof(float2) * n));
    DDH_CUDA(cudaMemcpy(d, h.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    g_twiddle[dev][s] = d;
    g_configured[dev][s] = true;
  }
  *tw = g_twiddle[dev][s];
  return DDH_OK;
}

int64_t aperture_limit(float d) { return static_cast<int64_t>(std::floor(static_cast<double>(d) * d)); }

int64_t aperture_count(int n, int64_t lim) {
  int64_t c = 0;
  for (int y = 0; y < n; ++y)
    for (int x = 0; x < n; ++x) {
      const int64_t dy = 2 * y - (n - 1), dx = 2 * x - (n - 1);
      if (dx * dx + dy * dy <= lim) ++c;
    }
  return c;
}

// The pupil's box in G x G tiles, from the integer pupil test: a column x holds pupil pixels iff
// (2x - (n-1))^2 + min_y (2y - (n-1))^2 <= ap_lim (the box is square, the pupil centred).
void tile_box(int n, int64_t ap_lim, int gs, int* t_lo, int* nt) {
  int64_t miny = INT64_MAX;
  for (int y = 0; y < n; ++y) miny = std::min<int64_t>(miny, int64_t(2 * y - (n - 1)) * (2 * y - (n - 1)));
  int lo = n, hi = -1;
  for (int x = 0; x < n; ++x) {
    const int64_t dx = 2 * x - (n - 1);
    if (dx * dx + miny <= ap_lim) {
      lo = std::min(lo, x);
      hi = std::max(hi, x);
    }
  }
  *t_lo = hi >= lo ? lo >> gs : 0;
  *nt = hi >= lo ? (hi >> gs) - *t_lo + 1 : 0;
}

int validate(const ddh_params* p) {
  if (p == nullptr || !supported_n(p->n)) return DDH_EINVAL;
  if (!(p->aperture_diam > 0.f && p->aperture_diam <= static_cast<float>(p->n))) return DDH_EINVAL;
  if (!(p->lambda >= 0.f && p->lambda <= 1.f && p->alpha >= 0.f && std::isfinite(p->alpha))) return DDH_EINVAL;
  if (p->n_k < 1 || p->n_k > 1024) return DDH_EINVAL;
  if (!(p->noise_var > 0.f && std::isfinite(p->noise_var))) return DDH_EINVAL;
  if (!(p->prior_p >= 1.f && p->prior_p < 2.f)) return DDH_EINVAL;
  if (p->prior_q != 2.f) return DDH_EINVAL;
  if (!(p->prior_T > 0.f && p->prior_sigma > 0.f && std::isfinite(p->prior_T) && std::isfinite(p->prior_sigma)))
    return DDH_EINVAL;
  if (!(p->r_floor > 0.f && std::isfinite(p->r_floor))) return DDH_EINVAL;
  if (p->tilt_mode != 0 && p->tilt_mode != 1) return DDH_EINVAL;
  if (p->phase_block != 1 && p->phase_block != 2 && p->phase_block != 4) return DDH_EINVAL;
  if (!(p->phase_prior >= 0.f && std::isfinite(p->phase_prior))) return DDH_EINVAL;
  if (p->phase_sweeps < 0 || p->phase_sweeps > 16) return DDH_EINVAL;
  if (p->noise_update != 0 && p->noise_update != 1) return DDH_EINVAL;
  if (p->phase_prior > 0.f && (p->phase_block == 1 || p->n_k != 1)) return DDH_EINVAL;
  if (p->exec_path < DDH_PATH_DEFAULT || p->exec_path > DDH_PATH_STAGED) return DDH_EINVAL;
  if (p->exec_path == DDH_PATH_CLUSTER && !cluster_n(p->n)) return DDH_EINVAL;
  if (staged_path(*p) && !staged_n(p->n)) return DDH_EINVAL;
  if (p->phase_prior > 0.f) {  // the prior's tile box must fit the post kernel
    int t_lo = 0, nt = 0;
    tile_box(p->n, aperture_limit(p->aperture_diam), p->phase_block == 4 ? 2 : 1, &t_lo, &nt);
    if (nt > ddh::kPostMaxTiles) return DDH_EINVAL;
  }
  return DDH_OK;
}

bool aux_needed(const ddh_params& p) { return p.phase_prior > 0.f || p.noise_update != 0; }

// The side buffer of the prior / sigma^2 M-steps: allocated when first needed; sigma^2 in use
// restarts at `nv` (stream-ordered).
int aux_reset(ddh_state* s, float nv) {
  if (!aux_needed(s->prm)) return DDH_OK;
  if (s->aux == nullptr) {
    DDH_CUDA(cudaMalloc(&s->aux, sizeof(float) * ddh::aux_floats(s->prm.n)));
    DDH_CUDA(cudaMemsetAsync(s->aux, 0, sizeof(float) * ddh::aux_floats(s->prm.n), s->stream));
  }
  const float h[2] = {nv, 0.f};
  DDH_CUDA(cudaMemcpyAsync(s->aux, h, sizeof(h), cudaMemcpyHostToDevice, s->stream));
  return DDH_OK;
}

// The post kernel's arguments for this state: the pupil's tile box from the integer pupil test.
ddh::PostArgs post_args(const ddh_state* s) {
  ddh::PostArgs a{};
  const int n = s->prm.n, gs = s->kp.g_shift;
  a.aux = s->aux;
  a.phi = s->phi;
  a.n = n;
  a.gs = gs;
  a.ap_lim = s->kp.ap_lim;
  a.ctas = s->staged ? n / 8 : n / ddh::kRowsPerCta;  // blocks that write partial sums
  a.prior = s->prm.phase_prior > 0.f ? 1 : 0;
  a.sweeps = s->prm.phase_sweeps > 0 ? s->prm.phase_sweeps : 2;
  a.noise_update = s->prm.noise_update;
  a.lam = s->prm.phase_prior;
  a.inv_ap_count = s->ap_count > 0 ? static_cast<float>(1.0 / static_cast<double>(s->ap_count)) : 0.f;
  a.inv_m = static_cast<float>(1.0 / (static_cast<double>(n) * n));
  a.nv_floor = 1e-6f;
  tile_box(n, a.ap_lim, gs, &a.t_lo, &a.nt);
  return a;
}

ddh::KParams derive(const ddh_params& p) {
  ddh::KParams k{};
  k.ap_lim = static_cast<int>(aperture_limit(p.aperture_diam));
  k.tilt_mode = p.tilt_mode;
  k.n_k = p.n_k;
  k.g_shift = p.phase_block == 4 ? 2 : p.phase_block == 2 ? 1 : 0;
  k.lam1 = static_cast<float>(1.0 - static_cast<double>(p.lambda));
  k.lam_alpha = static_cast<float>(static_cast<double>(p.lambda) * p.alpha);
  k.noise_var = p.noise_var;
  const double ts = static_cast<double>(p.prior_T) * p.prior_sigma;
  k.w0 = static_cast<float>(std::pow(ts, static_cast<double>(p.prior_p) - 2.0) *
                            std::pow(static_cast<double>(p.prior_sigma), -static_cast<double>(p.prior_p)));
  k.inv_tsig = static_cast<float>(1.0 / ts);
  k.q_minus_p = static_cast<float>(static_cast<double>(p.prior_q) - p.prior_p);
  k.q_over_p = static_cast<float>(static_cast<double>(p.prior_q) / p.prior_p);
  k.r_floor = p.r_floor;
  return k;
}

bool is_host_pointer(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

size_t image_bytes(int n) { return sizeof(float) * static_cast<size_t>(n) * n; }

int check_status(ddh_state* s) {
  unsigned h = 0;
  DDH_CUDA(cudaMemcpyAsync(&h, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
  DDH_CUDA(cudaStreamSynchronize(s->stream));
  if (h == 0) return DDH_OK;
  DDH_CUDA(cudaMemsetAsync(s->status, 0, sizeof(unsigned), s->stream));
  if ((h & ddh::kStatusTimeout) && s->staged)  // an abandoned persistent launch: fresh barrier words
    DDH_CUDA(cudaMemsetAsync(ddh::l2_stream_view(s->l2scratch, s->prm.n).bar, 0, 3 * sizeof(unsigned), s->stream));
  DDH_CUDA(cudaStreamSynchronize(s->stream));
  if (h & ddh::kStatusTimeout) return DDH_ETIMEOUT;
  return DDH_ENONFINITE;
}

ddh::FrameArgs frame_args(ddh_state* s, const void* y, float* trace) {
  ddh::FrameArgs f{};
  f.y = static_cast<const float2*>(y);
  f.r = s->r;
  f.phi = s->phi;
  f.status = s->status;
  f.trace = trace;
  return f;
}

ddh::L2Stream l2_view(ddh_state* s, const void* y) {
  ddh::L2Stream v = ddh::l2_stream_view(s->l2scratch, s->prm.n);
  v.y = static_cast<const float2*>(y);
  v.r = s->r;
  v.phi = s->phi;
  v.status = s->status;
  return v;
}

// A staged stream's entry `i` of a launch: its view, parameters and post-kernel side buffer.
void l2_put(ddh::L2Batch& lb, int i, ddh_state* s, const void* y) {
  lb.prm[i] = s->kp;
  lb.st[i] = l2_view(s, y);
  const bool aux = s->aux != nullptr && aux_needed(s->prm);
  lb.aux[i] = aux ? s->aux : nullptr;
  lb.aux_tiles[i] = aux && s->prm.phase_prior > 0.f ? 1 : 0;
}

// One step of `s` on frame `y`.  `y_host`: y is pinned host memory mapped into the device's
// address space (read in place by the kernel); `phi_copy`, `r_copy`: also write the frame's phi
// and r there (cluster path, neither post-step M-step on).
int enqueue(ddh_state* s, const void* y, float* trace, bool y_host = false, float* phi_copy = nullptr,
            float* r_copy = nullptr) {
  if (s == nullptr || y == nullptr) return DDH_EINVAL;
  if (reinterpret_cast<uintptr_t>(y) % 16 != 0) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  if (s->staged) {
    if (trace != nullptr || y_host || phi_copy != nullptr || r_copy != nullptr) return DDH_EINVAL;  // cluster path
    ddh::L2Batch lb{};
    l2_put(lb, 0, s, y);
    lb.tw = s->tw;
    lb.count = 1;
    DDH_CUDA(ddh::launch_step_l2(s->prm.n, g_schedule[s->device][n_slot(s->prm.n)], lb, s->kp.n_k, s->stream));
    if (lb.aux[0] != nullptr) DDH_CUDA(ddh::launch_post(post_args(s), s->stream));
    s->frame += 1;
    return DDH_OK;
  }
  ddh::StepBatch b{};
  b.prm[0] = s->kp;
  b.fa[0] = frame_args(s, y, trace);
  b.tw = s->tw;
  b.count = 1;
  if (s->aux != nullptr && aux_needed(s->prm)) {
    if (phi_copy != nullptr || r_copy != nullptr) return DDH_EINVAL;  // the post kernel changes phi later
    b.fa[0].aux = s->aux;
    b.fa[0].aux_tiles = s->prm.phase_prior > 0.f ? 1 : 0;
  }
  b.fa[0].y_host = y_host ? 1 : 0;
  b.fa[0].phi_copy = phi_copy;
  b.fa[0].r_copy = r_copy;
  DDH_CUDA(ddh::launch_step(s->prm.n, g_schedule[s->device][n_slot(s->prm.n)], b, s->stream, /*pdl=*/true));
  if (b.fa[0].aux != nullptr) DDH_CUDA(ddh::launch_post(post_args(s), s->stream));
  s->frame += 1;
  return DDH_OK;
}

// Enqueue one step of every state (all on `main`'s device): states are grouped by grid size
// and path, each group (chunks of kMaxBatch, or kMaxBatchL2 on the staged path) on its own side
// stream, forked from and joined back into `main`.  Frames come from `ys[i]` or, when `ytab` is
// set, from ytab[i] on the device (then the states of one launch must be consecutive).
int enqueue_batch(ddh_state* const* states, const void* const* ys, const float2* const* ytab, int count,
                  cudaStream_t main, int dev) {
  struct Group {
    int n;
    bool staged;
  };
  ddh_state* lb_states[ddh::kMaxBatchL2];  // the states of the staged launch being formed
  const Group order[kGroups] = {{512, true}, {256, true}, {128, true}, {32, false},
                                {64, false}, {128, false}, {256, false}};
  auto member = [&](int i, const Group& gr) { return states[i]->prm.n == gr.n && states[i]->staged == gr.staged; };
  // streams with the post-step M-steps keep the chained launches (their post kernel follows
  // each launch chunk)
  bool aux_staged = false;
  for (int i = 0; i < count; ++i) aux_staged |= states[i]->staged && states[i]->aux != nullptr && aux_needed(states[i]->prm);
  const bool persist = g_persistent[dev] != 0 && !aux_staged;
  int groups = 0;
  bool any_staged = false;
  for (const Group& gr : order)
    for (int i = 0; i < count; ++i)
      if (member(i, gr)) {
        if (gr.staged && persist) {
          if (!any_staged) ++groups;  // every staged stream shares the persistent branch
          any_staged = true;
        } else {
          ++groups;
        }
        break;
      }
  SideStreams* ss = nullptr;
  if (groups > 1) {
    int rc = side_streams(dev, &ss);
    if (rc != DDH_OK) return rc;
    DDH_CUDA(cudaEventRecord(ss->fork, main));
  }
  int g = 0;
  if (persist && any_staged) {
    cudaStream_t st = main;
    if (ss != nullptr) {
      st = ss->s[g];
      DDH_CUDA(cudaStreamWaitEvent(st, ss->fork, 0));
    }
    // the staged streams in runs of one grid size, as few persistent launches as the launch
    // limits allow (one when they are consecutive, share n_k and number at most 64)
    ddh::L2Persist lp{};
    auto flush = [&]() -> int {
      if (lp.b.count == 0) return DDH_OK;
      lp.bar = lp.b.st[0].bar;
      DDH_CUDA(ddh::launch_step_l2_persistent(lp, st));
      lp = ddh::L2Persist{};
      return DDH_OK;
    };
    int prev = -2;
    for (int i = 0; i < count; ++i) {
      ddh_state* s = states[i];
      if (!s->staged) continue;
      if (lp.b.count > 0 && (s->kp.n_k != lp.n_k || lp.b.count == ddh::kMaxBatchL2 ||
                             (ytab != nullptr && prev != i - 1) ||
                             (lp.n[lp.groups - 1] != s->prm.n && lp.groups == ddh::kPersistGroups))) {
        const int rc = flush();
        if (rc != DDH_OK) return rc;
      }
      if (lp.b.count == 0) {
        lp.b.ytab = ytab;
        lp.b.ytab_base = i;
        lp.n_k = s->kp.n_k;
      }
      if (lp.groups == 0 || lp.n[lp.groups - 1] != s->prm.n) {
        lp.first[lp.groups] = lp.b.count;
        lp.count[lp.groups] = 0;
        lp.n[lp.groups] = s->prm.n;
        lp.tw[lp.groups] = s->tw;
        ++lp.groups;
      }
      l2_put(lp.b, lp.b.count, s, ys != nullptr ? ys[i] : nullptr);
      ++lp.b.count;
      ++lp.count[lp.groups - 1];
      prev = i;
    }
    const int rc = flush();
    if (rc != DDH_OK) return rc;
    if (ss != nullptr) {
      DDH_CUDA(cudaEventRecord(ss->join[g], st));
      DDH_CUDA(cudaStreamWaitEvent(main, ss->join[g], 0));
    }
    ++g;
  }
  for (const Group& gr : order) {
    if (persist && gr.staged) continue;
    const int n = gr.n;
    int members = 0;
    for (int i = 0; i < count; ++i) members += member(i, gr) ? 1 : 0;
    if (members == 0) continue;
    cudaStream_t st = main;
    if (ss != nullptr) {
      st = ss->s[g];
      DDH_CUDA(cudaStreamWaitEvent(st, ss->fork, 0));
    }
    const int sched = g_schedule[dev][n_slot(n)];
    if (gr.staged) {
      ddh::L2Batch lb{};
      ddh::PostBatch pb{};  // the chunk's streams with the tile-phase prior or the sigma^2 M-step
      lb.ytab = ytab;
      lb.count = 0;
      auto flush = [&]() -> int {  // the chunk's step, then the post kernels of its aux streams
        DDH_CUDA(ddh::launch_step_l2(n, sched, lb, lb.prm[0].n_k, st));
        pb.count = 0;
        for (int j = 0; j < lb.count; ++j) {
          if (lb.aux[j] == nullptr) continue;
          pb.a[pb.count++] = post_args(lb_states[j]);
          if (pb.count == ddh::kMaxBatch) {
            DDH_CUDA(ddh::launch_post_batch(pb, st));
            pb.count = 0;
          }
        }
        if (pb.count > 0) DDH_CUDA(ddh::launch_post_batch(pb, st));
        lb.count = 0;
        return DDH_OK;
      };
      for (int i = 0; i < count; ++i) {
        ddh_state* s = states[i];
        if (!member(i, gr)) continue;
        const bool aux = s->aux != nullptr && aux_needed(s->prm);
        // one EM-iteration count per launch, and either all or none of its streams with the
        // post-step side buffer
        if (lb.count > 0 && (s->kp.n_k != lb.prm[0].n_k || aux != (lb.aux[0] != nullptr))) {
          const int rc = flush();
          if (rc != DDH_OK) return rc;
        }
        if (lb.count == 0) lb.ytab_base = i;
        l2_put(lb, lb.count, s, ys != nullptr ? ys[i] : nullptr);
        lb_states[lb.count] = s;
        lb.tw = s->tw;
        ++lb.count;
        const bool next_same = i + 1 < count && member(i + 1, gr);
        if (lb.count == staged_chunk(dev, n) || (ytab != nullptr && !next_same)) {
          const int rc = flush();
          if (rc != DDH_OK) return rc;
        }
      }
      if (lb.count > 0) {
        const int rc = flush();
        if (rc != DDH_OK) return rc;
      }
    } else {
      ddh::StepBatch b{};
      ddh::PostBatch pb{};  // the chunk's streams with the tile-phase prior or the sigma^2 M-step
      b.ytab = ytab;
      b.count = 0;
      auto flush = [&]() -> int {
        DDH_CUDA(ddh::launch_step(n, sched, b, st));
        if (pb.count > 0) DDH_CUDA(ddh::launch_post_batch(pb, st));
        b.count = 0;
        pb.count = 0;
        return DDH_OK;
      };
      for (int i = 0; i < count; ++i) {
        ddh_state* s = states[i];
        if (!member(i, gr)) continue;
        if (b.count == 0) b.ytab_base = i;  // ytab rows of one launch must be consecutive
        b.prm[b.count] = s->kp;
        b.fa[b.count] = frame_args(s, ys != nullptr ? ys[i] : nullptr, nullptr);
        if (s->aux != nullptr && aux_needed(s->prm)) {
          b.fa[b.count].aux = s->aux;
          b.fa[b.count].aux_tiles = s->prm.phase_prior > 0.f ? 1 : 0;
          pb.a[pb.count++] = post_args(s);
        }
        b.tw = s->tw;
        ++b.count;
        const bool next_same = i + 1 < count && member(i + 1, gr);
        if (b.count == ddh::kMaxBatch || (ytab != nullptr && !next_same)) {
          const int rc = flush();
          if (rc != DDH_OK) return rc;
        }
      }
      if (b.count > 0) {
        const int rc = flush();
        if (rc != DDH_OK) return rc;
      }
    }
    if (ss != nullptr) {
      DDH_CUDA(cudaEventRecord(ss->join[g], st));
      DDH_CUDA(cudaStreamWaitEvent(main, ss->join[g], 0));
    }
    ++g;
  }
  return DDH_OK;
}

struct CkptHeader {
  uint32_t magic;
  uint32_t version;
  ddh_params prm;
  int64_t frame;
  float noise_est;  // the running sigma^2 estimate (noise_update), else noise_var
  float pad;
};
constexpr uint32_t kMagic = 0x31484444u;  // "DDH1"


}  // namespace

int ddh_internal_cuda_fail(cudaError_t e) { return cuda_fail(e); }

int ddh_internal_state_info(const ddh_state* s, const ddh_params** prm, const void** twiddle, void** stream,
                            int* device) {
  if (s == nullptr) return DDH_EINVAL;
  *prm = &s->prm;
  *twiddle = s->tw;
  *stream = s->stream;
  *device = s->device;
  return DDH_OK;
}

void ddh_internal_set_error(const char* msg) { std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s", msg); }

size_t ddh_internal_state_bytes(const ddh_params* p) {
  if (p == nullptr || !supported_n(p->n)) return 0;
  const size_t img = image_bytes(p->n);
  // r, phi, 2-image staging buffer, status and scalar words (+ the L2-staged working images)
  return 4 * img + 512 + (staged_path(*p) ? ddh::l2_scratch_bytes(p->n) : 0);
}

int ddh_internal_backward_check(const ddh_state* s, const void* y, const float* trace) {
  const char* why = nullptr;
  if (s == nullptr)
    why = "frame-step adjoint: null state";
  else if (s->prm.n_k != 1 || s->prm.phase_block != 1)
    why = "frame-step adjoint: only one EM iteration per frame with the per-pixel phase is differentiated";
  else if (s->staged)
    why = "frame-step adjoint: grids up to 256 x 256 on the cluster path only";
  else if (aux_needed(s->prm))
    why = "frame-step adjoint: no adjoint through the tile-phase prior or the sigma^2 M-step";
  else if (y == nullptr || reinterpret_cast<uintptr_t>(y) % 16 != 0)
    why = "frame-step adjoint: frame pointer null or not 16-byte aligned";
  else if (trace == nullptr || reinterpret_cast<uintptr_t>(trace) % 8 != 0)
    why = "frame-step adjoint: trace pointer null or not 8-byte aligned";
  if (why == nullptr) return DDH_OK;
  ddh_internal_set_error(why);
  return DDH_EINVAL;
}

extern "C" {

int ddh_version(void) { return kVersion; }

const char* ddh_last_cuda_error(void) { return g_cuda_err; }

const char* ddh_strerror(int code) {
  switch (code) {
    case DDH_OK: return "ok";
    case DDH_EINVAL: return "invalid argument";
    case DDH_ENOMEM: return "device allocation failed";
    case DDH_ECUDA: return "CUDA runtime error";
    case DDH_ETIMEOUT: return "bounded device wait expired; frame dropped";
    case DDH_ENONFINITE: return "frame has a non-finite entry or zero variance; frame dropped";
    case DDH_EBUDGET: return "memory budget exceeded";
    default: return "unknown error";
  }
}

int ddh_default_params(ddh_params* p, int n, float aperture_diam, float snr) {
  if (p == nullptr || !supported_n(n) || !(aperture_diam > 0.f) || !(snr >= 0.f)) return DDH_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->n = n;
  p->aperture_diam = aperture_diam;
  p->lambda = 0.45f;
  p->alpha = 0.025f;
  p->n_k = 1;
  const double f = static_cast<double>(aperture_count(n, aperture_limit(aperture_diam))) /
                   (static_cast<double>(n) * n);
  p->noise_var = static_cast<float>(1.0 / (1.0 + f * snr));
  p->prior_p = 1.1f;
  p->prior_q = 2.0f;
  p->prior_T = 1.0f;
  p->prior_sigma = 0.1f;
  p->r_floor = 1e-10f;
  p->tilt_mode = 1;
  p->phase_block = 1;
  p->phase_prior = 0.f;
  p->phase_sweeps = 2;
  p->noise_update = 0;
  return DDH_OK;
}

int ddh_static_params(ddh_params* p, int n, float aperture_diam, float snr, int reset_every) {
  const int rc = ddh_default_params(p, n, aperture_diam, snr);
  if (rc != DDH_OK) return rc;
  if (reset_every < 1 || reset_every > 1024) return DDH_EINVAL;
  p->lambda = 1.f;
  p->alpha = 1.f;
  p->n_k = reset_every;
  p->tilt_mode = 0;
  return DDH_OK;
}

int ddh_tracking_params(ddh_params* p, int n, float aperture_diam, float snr) {
  const int rc = ddh_default_params(p, n, aperture_diam, snr);
  if (rc != DDH_OK) return rc;
  p->phase_block = 2;
  p->phase_prior = 10.f;
  p->prior_sigma = 0.03f;
  p->alpha = 0.0125f;
  return DDH_OK;
}

int ddh_init(ddh_state** out, const ddh_params* p, void* cuda_stream) {
  if (out == nullptr) return DDH_EINVAL;
  *out = nullptr;
  int rc = validate(p);
  if (rc != DDH_OK) return rc;
  int dev = 0;
  DDH_CUDA(cudaGetDevice(&dev));
  const float2* tw = nullptr;
  const bool staged = staged_path(*p);
  rc = device_setup(dev, p->n, &tw, staged);
  if (rc != DDH_OK) return rc;
  ddh_state* s = new ddh_state{};
  s->staged = staged;
  s->prm = *p;
  s->kp = derive(*p);
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->device = dev;
  s->tw = tw;
  s->ap_count = aperture_count(p->n, aperture_limit(p->aperture_diam));
  const size_t img = image_bytes(p->n);
  cudaError_t e = cudaMalloc(&s->r, img);
  if (e == cudaSuccess) e = cudaMalloc(&s->phi, img);
  if (e == cudaSuccess) e = cudaMalloc(&s->status, 256);
  if (e == cudaSuccess) e = cudaMalloc(&s->ystage, 2 * img);
  if (e == cudaSuccess) e = cudaMalloc(&s->scalar, 256);
  if (e == cudaSuccess && staged) e = cudaMalloc(&s->l2scratch, ddh::l2_scratch_bytes(p->n));
  if (e == cudaSuccess && staged)  // the frame flag and the grid-barrier words start at zero
    e = cudaMemsetAsync(ddh::l2_stream_view(s->l2scratch, p->n).flag, 0, 256, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->r, 0, img, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->phi, 0, img, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->status, 0, 256, s->stream);
  if (e != cudaSuccess) {
    const int code = cuda_fail(e);
    ddh_free(s);
    return code;
  }
  rc = aux_reset(s, p->noise_var);
  if (rc != DDH_OK) {
    ddh_free(s);
    return rc;
  }
  *out = s;
  return DDH_OK;
}

size_t ddh_trace_floats(int n) { return static_cast<size_t>(n) * n * 8 + 8; }

int ddh_step(ddh_state* s, const void* y) {
  DdhNvtxRange r("ddh_step");
  return enqueue(s, y, nullptr);
}

int ddh_step_trace(ddh_state* s, const void* y, float* trace) {
  DdhNvtxRange nv("ddh_step_trace");
  if (trace == nullptr) return DDH_EINVAL;
  return enqueue(s, y, trace);
}

// The device address of pinned, mapped host memory (cudaHostAlloc / cudaHostRegister), or null.
static void* mapped_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Host frames in place: where both buffers are pinned and mapped, the step kernel reads the frame
// and writes phi over the CPU-GPU link itself (no staging copies, one launch per frame).
static bool zero_copy(const ddh_state* s, const void* y_host, float* phi_host, const void** yd, float** pd) {
  if (s->staged || aux_needed(s->prm)) return false;
  *yd = mapped_host(y_host);
  *pd = static_cast<float*>(mapped_host(phi_host));
  return *yd != nullptr && *pd != nullptr && reinterpret_cast<uintptr_t>(*yd) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(*pd) % 16 == 0;
}

static int host_async_setup(ddh_state* s) {
  if (s->cin != nullptr) return DDH_OK;
  int prio = 0;
  DDH_CUDA(cudaStreamGetPriority(s->stream, &prio));
  DDH_CUDA(cudaMalloc(&s->hstage2, 2 * image_bytes(s->prm.n)));
  for (int i = 0; i < 2; ++i) {
    DDH_CUDA(cudaEventCreateWithFlags(&s->ev_in[i], cudaEventDisableTiming));
    DDH_CUDA(cudaEventCreateWithFlags(&s->ev_used[i], cudaEventDisableTiming));
  }
  for (cudaEvent_t& e : s->ev_done) DDH_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  DDH_CUDA(cudaStreamCreateWithPriority(&s->cin, cudaStreamNonBlocking, prio));
  return DDH_OK;
}

int ddh_step_host_async(ddh_state* s, const void* y_host, float* phi_host_out, int64_t* ticket) {
  DdhNvtxRange nv("ddh_step_host_async");
  if (s == nullptr || y_host == nullptr || phi_host_out == nullptr || ticket == nullptr) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  int rc = host_async_setup(s);
  if (rc != DDH_OK) return rc;
  const void* yd = nullptr;
  float* pd = nullptr;
  if (zero_copy(s, y_host, phi_host_out, &yd, &pd)) {
    rc = enqueue(s, yd, nullptr, true, pd);
    if (rc != DDH_OK) return rc;
    DDH_CUDA(cudaEventRecord(s->ev_done[s->hcount & 7], s->stream));
    *ticket = s->hcount++;
    return DDH_OK;
  }
  const size_t img = image_bytes(s->prm.n);
  const int slot = static_cast<int>(s->hcount & 1);
  float2* stage = slot == 0 ? s->ystage : s->hstage2;
  // the copy into a slot waits for the step that read it last (frame hcount - 2)
  DDH_CUDA(cudaStreamWaitEvent(s->cin, s->ev_used[slot], 0));
  DDH_CUDA(cudaMemcpyAsync(stage, y_host, 2 * img, cudaMemcpyHostToDevice, s->cin));
  DDH_CUDA(cudaEventRecord(s->ev_in[slot], s->cin));
  DDH_CUDA(cudaStreamWaitEvent(s->stream, s->ev_in[slot], 0));
  rc = enqueue(s, stage, nullptr);
  if (rc != DDH_OK) return rc;
  DDH_CUDA(cudaEventRecord(s->ev_used[slot], s->stream));
  // phi leaves on the state's stream, before the next step can overwrite it
  DDH_CUDA(cudaMemcpyAsync(phi_host_out, s->phi, img, cudaMemcpyDeviceToHost, s->stream));
  DDH_CUDA(cudaEventRecord(s->ev_done[s->hcount & 7], s->stream));
  *ticket = s->hcount++;
  return DDH_OK;
}

int ddh_host_wait(ddh_state* s, int64_t ticket) {
  if (s == nullptr || ticket < 0 || ticket >= s->hcount) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  // the slot holds this frame's event or a later frame's, which completes after it
  DDH_CUDA(cudaEventSynchronize(s->ev_done[ticket & 7]));
  return DDH_OK;
}

int ddh_step_host(ddh_state* s, const void* y_host, float* phi_host_out) {
  DdhNvtxRange nv("ddh_step_host");
  if (s == nullptr || y_host == nullptr || phi_host_out == nullptr) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  const void* yd = nullptr;
  float* pd = nullptr;
  if (zero_copy(s, y_host, phi_host_out, &yd, &pd)) {
    const int rc = enqueue(s, yd, nullptr, true, pd);
    if (rc != DDH_OK) return rc;
    return check_status(s);
  }
  const size_t img = image_bytes(s->prm.n);
  DDH_CUDA(cudaMemcpyAsync(s->ystage, y_host, 2 * img, cudaMemcpyHostToDevice, s->stream));
  int rc = enqueue(s, s->ystage, nullptr);
  if (rc != DDH_OK) return rc;
  DDH_CUDA(cudaMemcpyAsync(phi_host_out, s->phi, img, cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

static int copy_out(const ddh_state* cs, const float* src, float* out) {
  ddh_state* s = const_cast<ddh_state*>(cs);
  if (s == nullptr || out == nullptr) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  DDH_CUDA(cudaMemcpyAsync(out, src, image_bytes(s->prm.n), cudaMemcpyDefault, s->stream));
  if (is_host_pointer(out)) return check_status(s);
  return DDH_OK;
}

int ddh_phase(const ddh_state* s, float* out) { return s ? copy_out(s, s->phi, out) : DDH_EINVAL; }
int ddh_reflectance(const ddh_state* s, float* out) { return s ? copy_out(s, s->r, out) : DDH_EINVAL; }

int ddh_set_state(ddh_state* s, const float* r, const float* phi, int64_t frame_index) {
  if (s == nullptr || r == nullptr || phi == nullptr || frame_index < 0) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  const size_t img = image_bytes(s->prm.n);
  DDH_CUDA(cudaMemcpyAsync(s->r, r, img, cudaMemcpyDefault, s->stream));
  DDH_CUDA(cudaMemcpyAsync(s->phi, phi, img, cudaMemcpyDefault, s->stream));
  if (is_host_pointer(r) || is_host_pointer(phi)) DDH_CUDA(cudaStreamSynchronize(s->stream));
  s->frame = frame_index;
  return aux_reset(s, s->prm.noise_var);
}

int64_t ddh_frame_index(const ddh_state* s) { return s ? s->frame : -1; }

int ddh_set_params(ddh_state* s, const ddh_params* p) {
  if (s == nullptr || p == nullptr || validate(p) != DDH_OK || p->n != s->prm.n) return DDH_EINVAL;
  if (staged_path(*p) != s->staged) return DDH_EINVAL;  // the path is fixed for the state's lifetime
  DDH_ON_DEVICE(s->device);
  s->prm = *p;
  s->kp = derive(*p);
  s->ap_count = aperture_count(p->n, aperture_limit(p->aperture_diam));
  return aux_reset(s, p->noise_var);
}

int ddh_selftest_wait(ddh_state* s, double limit_s) {
  if (s == nullptr || !(limit_s > 0.0) || limit_s > 1.0) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  DDH_CUDA(ddh::launch_wait_selftest(s->status, static_cast<uint64_t>(limit_s * 1e9), s->stream));
  return check_status(s);
}

int ddh_noise_estimate(ddh_state* s, float* out) {
  if (s == nullptr || out == nullptr) return DDH_EINVAL;
  if (s->aux == nullptr || !aux_needed(s->prm) || !s->prm.noise_update) {
    *out = s->prm.noise_var;
    return DDH_OK;
  }
  DDH_ON_DEVICE(s->device);
  float h = 0.f;
  DDH_CUDA(cudaMemcpyAsync(&h, s->aux, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
  DDH_CUDA(cudaStreamSynchronize(s->stream));
  *out = h;
  return DDH_OK;
}
void* ddh_state_stream(const ddh_state* s) { return s ? static_cast<void*>(s->stream) : nullptr; }

int ddh_strehl(ddh_state* s, const float* phi_true_dev, float* out) {
  if (s == nullptr || phi_true_dev == nullptr || out == nullptr) return DDH_EINVAL;
  if (!cluster_n(s->prm.n)) {
    if (s->prm.n != 512 || s->l2scratch == nullptr) return DDH_EINVAL;
    // 512 x 512: a row and a column pass through the stream's first scratch image (scratch
    // between steps), the maximum gathered as float bits in the stream's scalar
    DDH_ON_DEVICE(s->device);
    ddh::StrehlL2Args a{};
    a.phi_est = s->phi;
    a.phi_true = phi_true_dev;
    a.work = ddh::l2_stream_view(s->l2scratch, s->prm.n).fa;
    a.max_bits = reinterpret_cast<unsigned*>(s->scalar);
    a.tw = s->tw;
    a.ap_lim = s->kp.ap_lim;
    DDH_CUDA(cudaMemsetAsync(s->scalar, 0, sizeof(float), s->stream));
    DDH_CUDA(ddh::launch_strehl_l2(s->prm.n, a, s->stream));
    float m = 0.f;
    DDH_CUDA(cudaMemcpyAsync(&m, s->scalar, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    const int rc = check_status(s);
    if (rc != DDH_OK) return rc;
    *out = m * static_cast<float>(1.0 / (static_cast<double>(s->ap_count) * s->ap_count));
    return DDH_OK;
  }
  DDH_ON_DEVICE(s->device);
  ddh::StrehlArgs a{};
  a.phi_est = s->phi;
  a.phi_true = phi_true_dev;
  a.out = s->scalar;
  a.tw = s->tw;
  a.ap_lim = s->kp.ap_lim;
  a.inv_ap_count2 = static_cast<float>(1.0 / (static_cast<double>(s->ap_count) * s->ap_count));
  DDH_CUDA(ddh::launch_strehl(s->prm.n, a, s->stream));
  DDH_CUDA(cudaMemcpyAsync(out, s->scalar, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

static int validate_batch(ddh_state* const* states, int count) {
  if (states == nullptr || count < 0) return DDH_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (states[i] == nullptr) return DDH_EINVAL;
    if (states[i]->stream != states[0]->stream || states[i]->device != states[0]->device) return DDH_EINVAL;
    for (int j = 0; j < i; ++j)
      if (states[j] == states[i]) return DDH_EINVAL;  // a stream advances once per batch
  }
  return DDH_OK;
}

int ddh_step_batch(ddh_state* const* states, const void* const* ys, int count) {
  DdhNvtxRange nv("ddh_step_batch");
  if (ys == nullptr) return DDH_EINVAL;
  int rc = validate_batch(states, count);
  if (rc != DDH_OK) return rc;
  if (count == 0) return DDH_OK;
  for (int i = 0; i < count; ++i)
    if (ys[i] == nullptr || reinterpret_cast<uintptr_t>(ys[i]) % 16 != 0) return DDH_EINVAL;
  DDH_ON_DEVICE(states[0]->device);
  rc = enqueue_batch(states, ys, nullptr, count, states[0]->stream, states[0]->device);
  if (rc != DDH_OK) return rc;
  for (int i = 0; i < count; ++i) states[i]->frame += 1;
  return DDH_OK;
}

// A captured batch: kSlots instances of the same graph, instance j reading its frame pointers
// from device table j.  Run k uses instance k % kSlots: the table is uploaded on a side copy
// stream (while the previous run's graph still executes) and the graph launch waits only for
// that copy, so no upload sits on the batch's stream between two steps.
constexpr int kBatchSlots = 4;
struct ddh_batch {
  int count;
  int device;
  cudaStream_t stream;
  cudaStream_t capture;
  cudaStream_t copy;
  std::vector<ddh_state*> states;
  const float2** ytab[kBatchSlots];     // device tables of frame pointers, one per instance
  const void** staging[kBatchSlots];    // pinned host copies of the tables
  cudaEvent_t copied[kBatchSlots];      // table j uploaded (copy stream)
  cudaEvent_t slot_done[kBatchSlots];   // instance j's last run finished (batch stream)
  int run;
  cudaGraph_t graph[kBatchSlots];
  cudaGraphExec_t exec[kBatchSlots];
};

int ddh_batch_free(ddh_batch* b) {
  if (b == nullptr) return DDH_OK;
  DdhDeviceGuard dg(b->device);
  cudaStreamSynchronize(b->stream);
  if (b->copy) cudaStreamSynchronize(b->copy);
  for (int j = 0; j < kBatchSlots; ++j) {
    if (b->exec[j]) cudaGraphExecDestroy(b->exec[j]);
    if (b->graph[j]) cudaGraphDestroy(b->graph[j]);
    cudaFree(const_cast<float2**>(b->ytab[j]));
    if (b->staging[j]) cudaFreeHost(b->staging[j]);
    if (b->copied[j]) cudaEventDestroy(b->copied[j]);
    if (b->slot_done[j]) cudaEventDestroy(b->slot_done[j]);
  }
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->copy) cudaStreamDestroy(b->copy);
  delete b;
  return DDH_OK;
}

int ddh_batch_create(ddh_batch** out, ddh_state* const* states, int count) {
  if (out == nullptr) return DDH_EINVAL;
  *out = nullptr;
  int rc = validate_batch(states, count);
  if (rc != DDH_OK) return rc;
  if (count == 0) return DDH_EINVAL;
  DDH_ON_DEVICE(states[0]->device);
  ddh_batch* b = new ddh_batch{};
  b->count = count;
  b->device = states[0]->device;
  b->stream = states[0]->stream;
  b->states.assign(states, states + count);
  cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->copy, cudaStreamNonBlocking);
  for (int j = 0; e == cudaSuccess && j < kBatchSlots; ++j) {
    e = cudaMalloc(&b->ytab[j], sizeof(float2*) * count);
    if (e == cudaSuccess) e = cudaMallocHost(&b->staging[j], sizeof(void*) * count);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied[j], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->slot_done[j], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    const int code = cuda_fail(e);
    ddh_batch_free(b);
    return code;
  }
  // capture one batched step (groups on concurrent branches) per table slot
  for (int j = 0; j < kBatchSlots && rc == DDH_OK; ++j) {
    e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      rc = cuda_fail(e);
      break;
    }
    rc = enqueue_batch(states, nullptr, b->ytab[j], count, b->capture, b->device);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
    b->graph[j] = g;
    if (rc == DDH_OK && e2 != cudaSuccess) rc = cuda_fail(e2);
    if (rc == DDH_OK) {
      e = cudaGraphInstantiate(&b->exec[j], b->graph[j], 0);
      if (e != cudaSuccess) rc = cuda_fail(e);
    }
  }
  if (rc != DDH_OK) {
    ddh_batch_free(b);
    return rc;
  }
  *out = b;
  return DDH_OK;
}

int ddh_batch_run(ddh_batch* b, const void* const* ys) {
  DdhNvtxRange nv("ddh_batch_run");
  if (b == nullptr || ys == nullptr) return DDH_EINVAL;
  for (int i = 0; i < b->count; ++i)
    if (ys[i] == nullptr || reinterpret_cast<uintptr_t>(ys[i]) % 16 != 0) return DDH_EINVAL;
  DDH_ON_DEVICE(b->device);
  const int j = b->run % kBatchSlots;
  // instance j's previous run has finished: its table and staging copy are free
  DDH_CUDA(cudaEventSynchronize(b->slot_done[j]));
  std::memcpy(b->staging[j], ys, sizeof(void*) * b->count);
  DDH_CUDA(cudaMemcpyAsync(const_cast<float2**>(b->ytab[j]), b->staging[j], sizeof(void*) * b->count,
                           cudaMemcpyHostToDevice, b->copy));
  DDH_CUDA(cudaEventRecord(b->copied[j], b->copy));
  DDH_CUDA(cudaStreamWaitEvent(b->stream, b->copied[j], 0));
  DDH_CUDA(cudaGraphLaunch(b->exec[j], b->stream));
  DDH_CUDA(cudaEventRecord(b->slot_done[j], b->stream));
  b->run += 1;
  for (ddh_state* s : b->states) s->frame += 1;
  return DDH_OK;
}

int ddh_step_backward(ddh_state* s, const void* y, const float* r_prev, const float* phi_prev, const float* trace,
                      const float* r_new, const float* r_bar, const float* phi_bar, float* r_prev_bar,
                      float* phi_prev_bar, float* grads, void* workspace, size_t workspace_bytes) {
  DdhNvtxRange nv("ddh_step_backward");
  if (s == nullptr || y == nullptr || r_prev == nullptr || phi_prev == nullptr || trace == nullptr ||
      r_new == nullptr || r_bar == nullptr || phi_bar == nullptr || r_prev_bar == nullptr ||
      phi_prev_bar == nullptr || grads == nullptr || workspace == nullptr)
    return DDH_EINVAL;
  int rc = ddh_internal_backward_check(s, y, trace);
  if (rc != DDH_OK) return rc;
  if (workspace_bytes < ddh_backward_workspace_bytes(s->prm.n) || reinterpret_cast<uintptr_t>(workspace) % 16 != 0) {
    ddh_internal_set_error("ddh_step_backward: workspace smaller than ddh_backward_workspace_bytes(n) or not "
                           "16-byte aligned");
    return DDH_EINVAL;
  }
  DDH_ON_DEVICE(s->device);
  return ddh_internal_step_backward(s->prm.n, &s->prm, s->tw, s->stream, y, r_prev, phi_prev, trace, r_new, r_bar,
                                    phi_bar, r_prev_bar, phi_prev_bar, grads, workspace);
}

size_t ddh_unrolled_workspace_bytes(int n) {
  const size_t bw = ddh_backward_workspace_bytes(n);
  if (bw == 0) return 0;
  const size_t M = static_cast<size_t>(n) * n;
  // backward workspace, one trace, two (r_bar, phi_bar) ping-pong pairs; 256-byte aligned parts
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(bw) + al(ddh_trace_floats(n) * sizeof(float)) + 4 * al(M * sizeof(float));
}

int ddh_unrolled_forward(ddh_state* s, int k_frames, const void* const* ys, float* const* r_ckpt,
                         float* const* phi_ckpt, float* const* traces) {
  DdhNvtxRange nv("ddh_unrolled_forward");
  if (s == nullptr || ys == nullptr || r_ckpt == nullptr || phi_ckpt == nullptr || k_frames < 1) return DDH_EINVAL;
  if (aux_needed(s->prm)) return DDH_EINVAL;  // no adjoint through the post-step M-steps
  DDH_ON_DEVICE(s->device);
  const size_t img = image_bytes(s->prm.n);
  for (int k = 0; k <= k_frames; ++k)
    if (r_ckpt[k] == nullptr || phi_ckpt[k] == nullptr) return DDH_EINVAL;
  // checkpoint 0 is the entry state; every step writes its outputs into the next checkpoint as
  // well as the state (no copies between the launches, which keeps them chained)
  DDH_CUDA(cudaMemcpyAsync(r_ckpt[0], s->r, img, cudaMemcpyDeviceToDevice, s->stream));
  DDH_CUDA(cudaMemcpyAsync(phi_ckpt[0], s->phi, img, cudaMemcpyDeviceToDevice, s->stream));
  for (int k = 0; k < k_frames; ++k) {
    float* tr = traces != nullptr ? traces[k] : nullptr;
    if (traces != nullptr && (tr == nullptr || reinterpret_cast<uintptr_t>(tr) % 8 != 0)) return DDH_EINVAL;
    const int rc = !s->staged ? enqueue(s, ys[k], tr, false, phi_ckpt[k + 1], r_ckpt[k + 1]) : DDH_EINVAL;
    if (rc != DDH_OK) return rc;
  }
  return DDH_OK;
}

int ddh_unrolled_backward(ddh_state* s, int k_frames, const void* const* ys, const float* const* r_ckpt,
                          const float* const* phi_ckpt, const float* const* traces, const float* r_bar,
                          const float* phi_bar, float* r0_bar, float* phi0_bar, float* grads, void* workspace,
                          size_t workspace_bytes) {
  DdhNvtxRange nv("ddh_unrolled_backward");
  if (s == nullptr || ys == nullptr || r_ckpt == nullptr || phi_ckpt == nullptr || r_bar == nullptr ||
      phi_bar == nullptr || r0_bar == nullptr || phi0_bar == nullptr || grads == nullptr || workspace == nullptr ||
      k_frames < 1)
    return DDH_EINVAL;
  const int n = s->prm.n;
  if (workspace_bytes < ddh_unrolled_workspace_bytes(n) || reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
    return DDH_EINVAL;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t M = static_cast<size_t>(n) * n, img = image_bytes(n);
  char* w = static_cast<char*>(workspace);
  void* bw = w;
  w += al(ddh_backward_workspace_bytes(n));
  float* trace = reinterpret_cast<float*>(w);
  w += al(ddh_trace_floats(n) * sizeof(float));
  float* rb[2] = {reinterpret_cast<float*>(w), reinterpret_cast<float*>(w + al(M * sizeof(float)))};
  w += 2 * al(M * sizeof(float));
  float* pb[2] = {reinterpret_cast<float*>(w), reinterpret_cast<float*>(w + al(M * sizeof(float)))};
  const float* rin = r_bar;
  const float* pin = phi_bar;
  for (int k = k_frames - 1; k >= 0; --k) {
    float* rout = k == 0 ? r0_bar : rb[k & 1];
    float* pout = k == 0 ? phi0_bar : pb[k & 1];
    const float* tr = traces != nullptr ? traces[k] : trace;
    int rc = DDH_OK;
    if (traces == nullptr) {  // recompute the frame's intermediates from its checkpoint
      rc = ddh_set_state(s, r_ckpt[k], phi_ckpt[k], k);
      if (rc == DDH_OK) rc = enqueue(s, ys[k], trace);
    } else if (tr == nullptr) {
      rc = DDH_EINVAL;
    }
    if (rc == DDH_OK)
      rc = ddh_step_backward(s, ys[k], r_ckpt[k], phi_ckpt[k], tr, r_ckpt[k + 1], rin, pin, rout, pout, grads, bw,
                             ddh_backward_workspace_bytes(n));
    if (rc != DDH_OK) return rc;
    rin = rout;
    pin = pout;
  }
  (void)img;
  if (traces != nullptr) return ddh_set_state(s, r_ckpt[0], phi_ckpt[0], 0);  // as after recomputing
  return DDH_OK;
}

int ddh_fft_schedule_count(int n) { return supported_n(n) ? ddh::schedule_count(n) : 0; }

int ddh_set_fft_schedule(int n, int schedule) {
  if (!supported_n(n) || schedule < 0 || schedule >= ddh::schedule_count(n)) return DDH_EINVAL;
  int dev = 0;
  DDH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  g_schedule[dev][n_slot(n)] = schedule;
  return DDH_OK;
}

int ddh_set_staged_chunk(int n, int chunk) {
  if (!staged_n(n) || chunk < 1 || chunk > ddh::kMaxBatchL2) return DDH_EINVAL;
  int dev = 0;
  DDH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  g_chunk[dev][n_slot(n)] = chunk;
  return DDH_OK;
}

int ddh_set_staged_persistent(int on) {
  if (on != 0 && on != 1) return DDH_EINVAL;
  int dev = 0;
  DDH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  g_persistent[dev] = on;
  return DDH_OK;
}

int ddh_get_staged_persistent(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DDH_ECUDA;
  return g_persistent[dev];
}

int ddh_get_staged_chunk(int n) {
  if (!staged_n(n)) return DDH_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DDH_ECUDA;
  return staged_chunk(dev, n);
}

int ddh_get_fft_schedule(int n) {
  if (!supported_n(n)) return DDH_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DDH_ECUDA;
  return g_schedule[dev][n_slot(n)];
}

int ddh_fft2(const void* in, void* out, int n, int inverse, void* cuda_stream) {
  if (in == nullptr || out == nullptr || !supported_n(n) || !cluster_n(n)) return DDH_EINVAL;
  int dev = 0;
  DDH_CUDA(cudaGetDevice(&dev));
  const float2* tw = nullptr;
  int rc = device_setup(dev, n, &tw);
  if (rc != DDH_OK) return rc;
  ddh::Fft2Args a{};
  a.in = static_cast<const float2*>(in);
  a.out = static_cast<float2*>(out);
  a.tw = tw;
  a.inverse = inverse ? 1 : 0;
  DDH_CUDA(ddh::launch_fft2(n, a, static_cast<cudaStream_t>(cuda_stream)));
  return DDH_OK;
}

int ddh_sync(ddh_state* s) {
  if (s == nullptr) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  return check_status(s);
}

size_t ddh_checkpoint_bytes(int n) {
  if (!supported_n(n)) return 0;
  return sizeof(CkptHeader) + 2 * image_bytes(n);
}

int ddh_save(ddh_state* s, void* buf, size_t bytes) {
  if (s == nullptr || buf == nullptr || bytes < ddh_checkpoint_bytes(s->prm.n)) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  CkptHeader h{};
  h.magic = kMagic;
  h.version = kVersion;
  h.prm = s->prm;
  h.frame = s->frame;
  h.noise_est = s->prm.noise_var;
  std::memcpy(buf, &h, sizeof(h));
  if (s->aux != nullptr && aux_needed(s->prm) && s->prm.noise_update)  // the running estimate
    DDH_CUDA(cudaMemcpyAsync(static_cast<char*>(buf) + offsetof(CkptHeader, noise_est), s->aux, sizeof(float),
                             cudaMemcpyDeviceToHost, s->stream));
  char* p = static_cast<char*>(buf) + sizeof(h);
  const size_t img = image_bytes(s->prm.n);
  DDH_CUDA(cudaMemcpyAsync(p, s->r, img, cudaMemcpyDeviceToHost, s->stream));
  DDH_CUDA(cudaMemcpyAsync(p + img, s->phi, img, cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

int ddh_load(ddh_state* s, const void* buf, size_t bytes) {
  if (s == nullptr || buf == nullptr || bytes < sizeof(CkptHeader)) return DDH_EINVAL;
  CkptHeader h{};
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kMagic || h.prm.n != s->prm.n || bytes < ddh_checkpoint_bytes(s->prm.n)) return DDH_EINVAL;
  if (validate(&h.prm) != DDH_OK || staged_path(h.prm) != s->staged) return DDH_EINVAL;
  DDH_ON_DEVICE(s->device);
  const char* p = static_cast<const char*>(buf) + sizeof(h);
  const size_t img = image_bytes(s->prm.n);
  DDH_CUDA(cudaMemcpyAsync(s->r, p, img, cudaMemcpyHostToDevice, s->stream));
  DDH_CUDA(cudaMemcpyAsync(s->phi, p + img, img, cudaMemcpyHostToDevice, s->stream));
  DDH_CUDA(cudaStreamSynchronize(s->stream));
  s->prm = h.prm;
  s->kp = derive(h.prm);
  s->ap_count = aperture_count(h.prm.n, aperture_limit(h.prm.aperture_diam));
  s->frame = h.frame;
  const int rc = aux_reset(s, h.noise_est);
  if (rc != DDH_OK) return rc;
  DDH_CUDA(cudaStreamSynchronize(s->stream));
  return DDH_OK;
}

int ddh_free(ddh_state* s) {
  if (s == nullptr) return DDH_OK;
  DdhDeviceGuard dg(s->device);
  cudaStreamSynchronize(s->stream);
  cudaFree(s->r);
  cudaFree(s->phi);
  cudaFree(s->status);
  cudaFree(s->ystage);
  cudaFree(s->scalar);
  cudaFree(s->l2scratch);
  cudaFree(s->aux);
  if (s->cin != nullptr) {
    cudaStreamSynchronize(s->cin);
    cudaStreamDestroy(s->cin);
    cudaFree(s->hstage2);
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(s->ev_in[i]);
      cudaEventDestroy(s->ev_used[i]);
    }
    for (cudaEvent_t e : s->ev_done) cudaEventDestroy(e);
  }
  delete s;
  return DDH_OK;
}

}  // extern "C"
