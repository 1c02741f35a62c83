// Kernel-side interface of libddh: launch parameter blocks and launchers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ddh {

constexpr int kMaxBatch = 32;   // streams per launch (kernel parameter block stays < 4 KB)
constexpr int kThreads = 512;   // 16 warps per CTA
constexpr int kRowsPerCta = 16; // local rows (cyclic) == slab columns per CTA

// status bits latched by the kernels in the per-stream device status word
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusTimeout = 2u;

// Method parameters in the form the kernels use (derived on the host from ddh_params).
struct KParams {
  int ap_lim;        // floor(d^2): pixel in pupil iff (2x-(N-1))^2 + (2y-(N-1))^2 <= ap_lim
  int tilt_mode;     // RemoveTipTilt on/off
  int n_k;           // EM iterations per frame
  int g_shift;       // log2 of the phase tile G; rows are dealt to CTAs in groups of G
  float lam1;        // 1 - lambda
  float lam_alpha;   // lambda * alpha
  float noise_var;   // sigma^2
  float w0;          // (T sigma_r)^(p-2) sigma_r^(-p)
  float inv_tsig;    // 1 / (T sigma_r)
  float q_minus_p;   // q - p
  float q_over_p;    // q / p
  float r_floor;
};

// One stream's frame: input, state (in/out), status word, optional trace output, optional
// side outputs for the post kernel (`aux`, below).
struct FrameArgs {
  const float2* y;
  float* r;
  float* phi;
  unsigned* status;
  float* trace;
  float* aux;      // null: sigma^2 from KParams, no side outputs
  int aux_tiles;   // 1: write the pupil tiles' sums (phase prior), 0: per-CTA residual partials
  int y_host;      // 1: y is pinned host memory mapped into the device's address space, read
                   //    with plain 16-byte loads (not TMA) over the CPU-GPU link
  float* phi_copy; // optional second destination of the frame's phi (device memory, or pinned
                   //    host memory mapped into the device's address space)
  float* r_copy;   // optional second destination of the frame's r (device memory)
};

// Per-stream side buffer of the tile-phase prior and sigma^2 M-steps (aux_floats(n) floats):
//   aux[0]                     sigma^2 in use: read by the step kernel after its dependency
//                              wait, replaced by the post kernel when sigma^2 is re-estimated
//   aux[1]                     1 when the step accepted the frame, 0 when it dropped it
//   aux[kAuxPart + 2k, + 1]    block k's sums (a cluster kernel's CTA k, or the k-th 8-row and
//                              8-column block of the L2-staged kernels; at most kAuxParts):
//                              pupil residual at the tile angles, sum of C
//   aux[kAuxTiles ...]         float4 per tile of the N/G x N/G grid (row-major), written for
//                              the tiles that hold a pupil pixel: (Re v_t, Im v_t, E_t, 0),
//                              v_t = sum a y~ conj(z), E_t = sum a (|y~|^2 + |z|^2)
constexpr int kAuxPart = 16;
constexpr int kAuxParts = 64;
constexpr int kAuxTiles = kAuxPart + 2 * kAuxParts;
constexpr int kPostMaxTiles = 128;  // the tile-phase prior's box: at most 128 x 128 tiles
inline size_t aux_floats(int n) { return kAuxTiles + size_t(4) * (n / 2) * (n / 2); }

struct PostArgs {
  float* aux;
  float* phi;
  int n, gs, ap_lim, ctas;    // grid, log2 tile, pupil limit, CTAs of the step kernel
  int prior, sweeps, noise_update;
  float lam;                  // precision of the tile-phase prior
  float inv_ap_count, inv_m;  // 1 / |P|, 1 / N^2
  float nv_floor;
  int t_lo, nt;               // the pupil tiles lie in [t_lo, t_lo + nt)^2
};

// The post kernel's arguments of a batch's streams (one 8-CTA cluster each, blockIdx.y).
struct PostBatch {
  PostArgs a[kMaxBatch];
  int count;
};

struct StepBatch {
  KParams prm[kMaxBatch];
  FrameArgs fa[kMaxBatch];
  const float2* tw;                  // twiddle table exp(-2 pi i t / N), t < N
  const float2* const* ytab;         // if set, stream i's frame is ytab[ytab_base + i]
  int ytab_base;
  int count;
};

// L2-staged path (grids beyond a cluster's shared memory, or any batch run for throughput):
// per-stream views of the global scratch the stages exchange data through.  A batch is cut
// into launch chunks of at most kMaxBatchL2 streams (the chunk size is a tuning knob).
constexpr int kMaxBatchL2 = 64;

struct L2Stream {
  const float2* y;
  float* r;
  float* phi;
  unsigned* status;
  float2* fa;     // row-major complex image (z rows for the phase step)
  float2* fb;     // column-major complex image (back-projection columns)
  float* r0;      // r-init (entry values of the ICD sweep)
  float* s;       // E|g|^2
  float* beta;    // 4 images of pair weights: E, S, SE, SW
  float* part;    // row-block statistics, then the combined statistics
  int* flag;      // frame dropped (non-finite or zero variance)
  unsigned* bar;  // grid-barrier words of a persistent launch led by this stream (zeroed at init)
};

struct L2Batch {
  KParams prm[kMaxBatchL2];
  L2Stream st[kMaxBatchL2];
  const float2* tw;
  const float2* const* ytab;
  int ytab_base;
  int count;
  float* aux[kMaxBatchL2];     // per stream: side buffer of the post-step M-steps (layout above), or null
  int aux_tiles[kMaxBatchL2];  // with aux: 1 = tile sums for the phase prior, 0 = residual partial sums
};

// One persistent launch for a whole staged batch: every stage of every stream, the stages
// separated by grid-wide barriers.  The streams of `b` come in up to kPersistGroups runs of
// one grid size each (group g: streams [first[g], first[g] + count[g]) of size n[g], twiddle
// table tw[g]); they share n_k.  `bar` points to three zeroed words (arrivals, generation,
// abort) that no other launch uses at the same time.
constexpr int kPersistGroups = 4;
struct L2Persist {
  L2Batch b;
  int groups;
  int first[kPersistGroups];
  int count[kPersistGroups];
  int n[kPersistGroups];
  const float2* tw[kPersistGroups];
  int n_k;
  unsigned* bar;
};
cudaError_t launch_step_l2_persistent(const L2Persist& p, cudaStream_t st);

size_t l2_scratch_bytes(int n);                    // per stream; 0 when n uses the cluster kernel
L2Stream l2_stream_view(void* scratch, int n);     // y, r, phi, status left for the caller
cudaError_t configure_l2(int n);
cudaError_t launch_step_l2(int n, int schedule, const L2Batch& b, int n_k, cudaStream_t st);

struct StrehlArgs {
  const float* phi_est;
  const float* phi_true;
  float* out;           // one float
  const float2* tw;
  int ap_lim;
  float inv_ap_count2;  // 1 / (sum a)^2
};

struct Fft2Args {
  const float2* in;
  float2* out;
  const float2* tw;
  int inverse;
};

// Launchers (return the CUDA error of the launch).  `n` selects the template instance.
// `pdl`: launch with programmatic stream serialization, so that the kernel's prologue (frame
// TMA, twiddles, frame statistics) overlaps the tail of the previous kernel on `st`.
cudaError_t launch_step(int n, int schedule, const StepBatch& b, cudaStream_t st, bool pdl = false);
cudaError_t launch_strehl(int n, const StrehlArgs& a, cudaStream_t st);
cudaError_t launch_fft2(int n, const Fft2Args& a, cudaStream_t st);
// Post-step kernel (one CTA; programmatic launch): prior-weighted tile-phase M-step and/or
// the sigma^2 M-step from the step kernel's side outputs.
cudaError_t launch_post(const PostArgs& a, cudaStream_t st);
cudaError_t launch_post_batch(const PostBatch& b, cudaStream_t st);
// One-time per-device function attributes (shared memory size, cluster size); also checks
// that a cluster of this shape can be resident.  Returns cudaSuccess or the failing error.
cudaError_t configure(int n, int* max_active_clusters);
size_t step_smem_bytes(int n);
int schedule_count(int n);  // FFT radix schedules available for grid n

}  // namespace ddh
