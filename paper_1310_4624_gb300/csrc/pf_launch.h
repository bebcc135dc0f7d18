// pf_launch.h -- kernel argument blocks and launchers shared by the C-ABI
// layer (pf_api.cu) and the kernels (pf_kernels.cu).  Internal to libpfarna.
#pragma once

#include <cuda_runtime.h>

#include "pf_device.cuh"

namespace pf {

struct InitArgs {
  const TrackParams* trk;
  const int4* tiles;   // (track, group, first slot, count) per tile
  int n_tiles;
  long long n_total;
  const float* user;   // 5 x n_total SoA or nullptr
  float4* pv;          // buffer read by step 0
  float* In;
};

struct FrameArgs {
  const TrackParams* trk;
  float* ypad;
  int* frame_of;       // per track: the track whose padded frame holds its frame this step
  int t0;              // first track of this launch
  int nt;              // tracks of this launch
  int R;
  const float* frames[MAX_FRAMES_PER_LAUNCH];
  // tracks given the same frame (same pointer, size and background) share
  // one padded copy: rep[y] is the track that blockIdx.y prepares, and
  // share[i] the track (absolute) whose copy track t0 + i reads
  short rep[MAX_FRAMES_PER_LAUNCH];
  int share[MAX_FRAMES_PER_LAUNCH];
};

struct FrameTableArgs {
  const TrackParams* trk;
  float* ypad;
  int R;
  const float* const* table;  // device: T_table x n_tracks frame pointers
  int T_table;
  int n_tracks;
  const TrackState* ts;
  DevState* ds;
  int* frame_of;              // set to the identity: every track reads its own copy
};

struct K1Args {
  const TrackParams* trk;
  const int4* tiles;
  int n_tiles;
  GroupState* grp;
  TrackState* ts;
  DevState* ds;
  float4* pv0;
  float4* pv1;
  float* I0;
  float* I1;
  uint32_t* anc;        // ancestors, two buffers of anc_stride by step parity: step k reads
                        // buffer (k + 1) & 1 (the previous step's) and resamples into buffer k & 1
  long long anc_stride;
  uint32_t* parent;     // ancestry records or nullptr
  int history;
  float* lw;            // log-weights; with carried weights, two buffers by step parity:
  float* lw1;           // step k writes lw (k even) or lw1 (k odd) and reads the other one
                        // (lw1 == lw when no track carries weights)
  float* tile_part;     // 8 floats per tile
  const float* ypad;
  const CUtensorMap* tmaps;  // one per track over its padded frame, or nullptr
  int* ring_next;            // two buffers (by step parity) of G_total: ring order of step k+1 (ARNA)
  int ring_stride;           // G_total
  int* ring;                 // ring order of each group's track (the global step's output)
  uint32_t* exo_next;        // two buffers (by step parity) of G_total: exchange offsets of step k+1
  HistRec* hist;
  GroupHist* ghist;
  int* tile_ctr;             // dynamic tile counter (zero at launch; the resampler resets it)
  int n_ring_blocks;         // leading blocks: next step's rings and exchange offsets, previous step's history
  int n_tracks;
  TrackParams p0;            // n_tracks == 1: a copy of trk[0]
  // n_tracks == 1 and raw_frame: the step reads the caller's frame (W x H
  // float32, row pitch W) directly, through zmap (TMA, zero fill outside)
  // or zraw, instead of the padded frame y = z - b.
  int raw_frame;
  const float* zraw;
  int test_withhold_copy;    // failure-detection test: issue no staging copy, so the bounded wait runs out
  int variants;              // 1: some track resamples by Alg. 1's test (groups may carry weights) or
                             // uses keyed send sets: launches the variants instance (frames prepared)
  uint4* keys_next;          // two buffers (by step parity) of G_total: keyed send-permutation keys of step k+1
  const int* frame_of;       // per track: the track whose padded frame to read this step, or nullptr (its own)
  // fused step (one persistent launch per step): the resampling chunks,
  // their code sums, the counters and the ready queue of resampling tasks
  int n_chunks;
  const int4* chunks;        // (track, global group, first slot in the group, items)
  const GroupDesc* gd;
  unsigned long long* chunk_q;  // per chunk: sum of weight codes, for Alg. 1's test sums of c and c^2,
                                // and the sum of the codes of the group's chunks before it
  unsigned int* sync;        // counters by step parity (FusedSync)
  unsigned int* rq;          // ready queue, two parities of 2 n_chunks entries: task + 1, 0 = not yet written
  QuantCoeffs qc;
  CUtensorMap zmap;
};

// Offsets of the fused step's counters in K1Args::sync, by step parity:
// per global group the tiles done and the chunks quantised, then the tile
// counter, CTAs that left, leading blocks done, and the ready queue's claim
// and publish positions.
struct FusedSync {
  int G_total;
  __host__ __device__ int pdone(int par, int gi) const { return par * G_total + gi; }
  __host__ __device__ int adone(int par, int gi) const { return 2 * G_total + par * G_total + gi; }
  __host__ __device__ int tile_ctr(int par) const { return 4 * G_total + par; }
  __host__ __device__ int exit_ctr(int par) const { return 4 * G_total + 2 + par; }
  __host__ __device__ int ring_done(int par) const { return 4 * G_total + 4 + par; }
  // claim position and publish position side by side (one 8-byte aligned
  // load reads both: the counters start 256-byte aligned and 4 G_total + 6
  // is even)
  __host__ __device__ int rq_head(int par) const { return 4 * G_total + 6 + 2 * par; }
  __host__ __device__ int rq_tail(int par) const { return 4 * G_total + 7 + 2 * par; }
  __host__ __device__ int count() const { return 4 * G_total + 10; }
};

struct GlobalArgs {
  const TrackParams* trk;
  TrackState* ts;
  GroupState* gs;
  int* ring;
  const int* ring_next;  // two buffers by step parity: ring of the next step, drawn by the propagate kernel
  int ring_stride;
  const uint32_t* exo_next;  // two buffers by step parity: exchange offsets of the next step
  HistRec* hist;
  GroupHist* ghist;
  int history;
  int finalize;  // 0: prepare step 0 only
  DevState* ds;
  int keep_k;    // 1: leave the step index to the caller (fused step: advanced when its launch ends)
};

struct ResampleArgs {
  const GroupDesc* gd;
  GroupState* gs;
  const float* tile_part;      // nullptr: no group estimate
  const float* lw;
  const float* lw1;            // filter step with carry: the weights are lw1 at odd steps (nullptr: always lw)
  uint32_t* anc;               // filter step: two buffers of anc_stride by step parity (step k writes k & 1)
  long long anc_stride;        // 0: a single output array
  unsigned long long* q_out;   // nullptr: not stored
  const uint32_t* u_arr;       // nullptr: GroupState::u
  int local_idx;               // 1: ancestors within the group
  QuantCoeffs qc;
  DevState* ds;
  int fuse_global;             // 1: the last group of a track to finish runs its global step;
                               // 2 (one track): an extra cluster after the groups' runs it instead,
                               // once every group has reported, so no group's merge waits behind it
  int n_groups;                // groups of the launch (the extra cluster, if any, comes after them)
  int lean;                    // 1: no group under Alg. 1's test and no codes stored (a filter step, or
                               // pf_resample without codes): the lean instance runs if every CTA's chunk
                               // also fits its registers
  int max_np;                  // the largest group of the launch (for that test)
  int* tile_ctr;               // propagate kernel's tile counter to reset, or nullptr
  GlobalArgs glob;             // (fuse_global) arguments of that step, finalize = 1
};

// pf_backward (pf_adjoint.cu)
struct ReplayArgs {
  const TrackParams* trk;
  const int4* tiles;
  int n_tiles;
  const uint32_t* parent;  // recorded ancestry
  int history;
  int k;
  const float4* pv_in;     // X_{k-1} (k >= 1)
  const float* I_in;
  float4* pv_out;          // X_k (read only at k = 0)
  float* I_out;
  float4* ck_pv;           // optional copy of X_k (checkpoint), or nullptr
  float* ck_I;
  int weights;             // 1: log-weights and per-tile (max, sum exp)
  const float* ypad;
  const double* lbar_prev; // lbar_{k-1} per global group (k >= 1)
  float* tile_part;
};

struct ReplayGroupArgs {
  const TrackParams* trk;
  const GroupDesc* gd;
  const float* tile_part;
  int k;
  int G_total;
  double* lam_hist;        // [k][global group]
  double* lbar_hist;
  double* logZ;            // per track, accumulated
  double* dlam;            // per global group: the reverse sweep's seed at the last step
  const float* seed;       // per track
  int last;
};

struct AdjointArgs {
  const TrackParams* trk;
  const int4* tiles;
  int n_tiles;
  const uint32_t* parent;
  int history;
  int k;
  const float4* pv;        // X_k
  const float* In;
  const float* ypad;
  const double* lbar_prev; // lbar_{k-1} (k >= 1)
  const double* lam_k;     // L_k
  const double* dlam_k;    // dL_k
  double* D;               // dL_{k-1} accumulator per global group
  float4* Cc_pv;           // state adjoint of X_k (read and cleared)
  float* Cc_I;
  float4* Cp_pv;           // state adjoint of X_{k-1} (accumulated)
  float* Cp_I;
  double* grad;            // per track x 5
};

cudaError_t launch_replay(const ReplayArgs& a, int R, int grid, cudaStream_t s);
cudaError_t launch_replay_groups(const ReplayGroupArgs& a, int n_tracks, int max_G, cudaStream_t s);
cudaError_t launch_adjoint(const AdjointArgs& a, int R, int grid, cudaStream_t s);
cudaError_t launch_adjoint_groups(double* dlam, double* D, int G_total, cudaStream_t s);
cudaError_t launch_grad_out(const double* g, const double* lz, float* out, double* lz_out, int n, cudaStream_t s);
// parents (T x n_total, row k = step k) into the replay's ancestry record;
// out-of-range indices are counted in *bad (not read or written past)
cudaError_t launch_set_replay(const TrackParams* trk, const int4* tiles, int n_tiles, const uint32_t* parents,
                              long long n_total, uint32_t* parent, int history, int T, int* bad, int grid,
                              cudaStream_t s);

cudaError_t launch_init(const InitArgs& a, int grid, cudaStream_t s);
// The step launchers take `pdl`: launch with programmatic stream
// serialization, so the kernel's CTAs may start while the previous kernel
// in the stream drains; every step kernel waits (griddepcontrol.wait) for
// that kernel's completion and memory before touching any buffer.
cudaError_t launch_frame_prep(const FrameArgs& a, int nt, int blocks_x, bool pdl, cudaStream_t s);
cudaError_t launch_frame_prep_table(const FrameTableArgs& a, int blocks_x, bool pdl, cudaStream_t s);
cudaError_t launch_propagate(const K1Args& a, int R, int grid, bool pdl, cudaStream_t s);
// The fused step: propagate + weight tiles, the per-group resampling and the
// global step in one persistent launch.
cudaError_t launch_fused_step(const K1Args& a, int R, int grid, bool pdl, cudaStream_t s);
cudaError_t fused_occupancy(int R, int* blocks_per_sm);
// threads: RS_THREADS, or RS_THREADS_SMALL (eight CTAs per SM, for batches of small groups)
cudaError_t launch_resample(const ResampleArgs& a, int n_groups, int cluster, bool pdl, cudaStream_t s,
                            int threads = RS_THREADS);
cudaError_t launch_global(const GlobalArgs& a, int n_tracks, cudaStream_t s);
cudaError_t launch_finish(const GlobalArgs& a, int n_tracks, cudaStream_t s);
// launch_finish, then x^ (n_tracks x 5) and log Z (n_tracks) stored through
// device addresses of page-locked host memory (either may be null); pdl:
// programmatic dependent launch behind the previous kernel
cudaError_t launch_finish_out(const GlobalArgs& a, int n_tracks, float* xhat, double* logZ, bool pdl,
                              cudaStream_t s);
cudaError_t launch_export_states(const float4* pv, const float* In, long long n, float* out, cudaStream_t s);
cudaError_t k1_occupancy(int R, int* blocks_per_sm);
const void* propagate_kernel(int R);

// Host helpers shared by the C-ABI entry points (defined in pf_api.cu).
QuantCoeffs resample_coeffs();             // weight-code coefficients
int resample_cluster_size(int Np);         // resampler cluster size for one group of Np
void set_handleless_error(const char* msg);  // text for pf_last_error(NULL)
// The no-allocation resampler's error word on the current device (defined
// in pf_noalloc.cu); PF_OK and *out set, or an error status.
int noalloc_error_word(const DevState** out);

}  // namespace pf
