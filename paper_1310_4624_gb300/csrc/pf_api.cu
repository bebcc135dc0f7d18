// pf_api.cu -- the C ABI declared in include/pfarna.h: validation, workspace
// layout, launch sequence of one filter step, and read-back.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <unordered_map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pfarna.h"
#include "pf_device.cuh"
#include "pf_launch.h"

using namespace pf;

struct pf_handle {
  int n_tracks = 0, history = 0, R = 5;
  std::vector<pf_track_config> cfg;
  std::vector<TrackParams> tp;
  long long N_total = 0;
  int G_total = 0, n_tiles = 0;
  int k1_grid = 1, rs_cluster = 1;
  int rs_threads = RS_THREADS;  // resampler CTA: RS_THREADS, or RS_THREADS_SMALL for small groups
  int steps_run = 0;
  int failed = 0;
  cudaStream_t last_stream = nullptr;
  // pf_step_host: the upload stream and, per staging slot, "copied" and
  // "read by its step" events (created on first use)
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_copied[2] = {nullptr, nullptr}, up_used[2] = {nullptr, nullptr};
  std::string err;
  QuantCoeffs qc{};
  // device pointers into the caller's workspace
  TrackParams* trk = nullptr;
  TrackState* ts = nullptr;
  GroupState* gs = nullptr;
  GroupDesc* gd = nullptr;
  int4* tiles = nullptr;
  int* frame_of = nullptr;  // per track: whose padded frame the step reads (tracks given the same frame share one)
  float4* pv[2] = {nullptr, nullptr};
  float* In[2] = {nullptr, nullptr};
  uint32_t* anc = nullptr;
  float* lw = nullptr;   // two buffers lw_stride(N_total) apart; with carry_any step k writes buffer k & 1, else buffer 0
  float* tile_part = nullptr;
  float* ypad = nullptr;
  HistRec* hist = nullptr;
  GroupHist* ghist = nullptr;
  int* ring = nullptr;
  int* ring_next = nullptr;
  uint32_t* exo_next = nullptr;
  uint4* keys_next = nullptr;  // two buffers (by step parity) of G_total: send-permutation keys of step k+1
  int* tile_ctr = nullptr;
  int n_ring_blocks = 0;  // leading blocks of the propagate kernel
  // fused step: task list, resampling chunks, their code sums, counters
  int4* chunks = nullptr;
  int n_chunks = 0;
  unsigned long long* chunk_q = nullptr;
  unsigned int* fsync = nullptr;
  unsigned int* rq = nullptr;  // ready queue, 2 parities x 2 n_chunks entries
  int fused_grid = 1;
  bool fused = false;  // PFARNA_FUSED=1 at pf_init: the whole step as one persistent launch
  bool global_cta = true;  // PFARNA_GLOBAL_CTA=0 at pf_init: the last group to report runs the global step
  bool finish_pending = false;  // the last step's estimate / history not yet written (k_finish)
  int max_G = 1;
  uint32_t* parent = nullptr;
  DevState* ds = nullptr;
  CUtensorMap* tmaps = nullptr;  // nullptr: frames read through L1 only
  // pf_backward buffers (present when every track records its ancestry)
  bool adjoint = false;
  int adj_slots = 0, adj_ckpts = 0;
  float4* rp_pv = nullptr;   // adj_slots x N_total (replay / segment states)
  float* rp_I = nullptr;
  float4* ck_pv = nullptr;   // adj_ckpts x N_total (checkpoints)
  float* ck_I = nullptr;
  float4* ca_pv[2] = {nullptr, nullptr};  // state adjoints
  float* ca_I[2] = {nullptr, nullptr};
  double* lam_hist = nullptr;   // history x G_total
  double* lbar_hist = nullptr;
  double* dlam = nullptr;       // G_total
  double* Dacc = nullptr;       // G_total
  double* grad = nullptr;       // n_tracks x 5
  double* logz_rp = nullptr;    // n_tracks
  float* seed = nullptr;        // n_tracks
  int* replay_bad = nullptr;    // pf_set_replay's count of out-of-range parents
  bool replay_invalid = false;  // a rejected pf_set_replay left the ancestry unusable
  // pf_graph_step: the captured step for one frame table
  cudaGraphExec_t graph = nullptr;
  const void* graph_table = nullptr;
  int graph_T = 0;
  int k1_occ = 1, sms = 1;
  bool pdl = true;  // programmatic dependent launch between the step kernels
  bool test_withhold_copy = false;  // PFARNA_TEST_WITHHOLD_COPY=1 at pf_init (failure-detection tests)
  bool carry_any = false;           // some track resamples by Alg. 1's test (PF_RESAMPLE_ESS)
  bool variants = false;            // carry_any, or some track uses PF_SEND_KEYED
  char* ws = nullptr;        // the workspace, its size, and the byte range of the TMA
  size_t ws_total = 0;       // descriptors in it (they hold this workspace's addresses)
  size_t tmap_off = 0, tmap_bytes = 0;
  unsigned long long cfg_sig = 0;  // signature of the configurations and history
  void* encode = nullptr;  // cuTensorMapEncodeTiled, or nullptr
  // kernel timing (pf_profile_enable / pf_profile_read)
  int prof = 0;
  std::vector<cudaEvent_t> ev[PF_KERNEL_COUNT];  // start, stop, start, stop, ...
  ~pf_handle() {
    for (auto& v : ev)
      for (cudaEvent_t e : v) cudaEventDestroy(e);
    if (graph) cudaGraphExecDestroy(graph);
    for (int i = 0; i < 2; ++i) {
      if (up_copied[i]) cudaEventDestroy(up_copied[i]);
      if (up_used[i]) cudaEventDestroy(up_used[i]);
    }
    if (up_stream) cudaStreamDestroy(up_stream);
  }
};

namespace {

thread_local std::string g_err;

// An NVTX range around an entry point (a no-op unless a profiler listens):
// profiler timelines show each pf_* call above the kernels it launched.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

pf_status fail(pf_handle* h, pf_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_err = msg;
  return st;
}

pf_status cuda_fail(pf_handle* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (h) h->failed = 1;
  return fail(h, PF_ERR_CUDA, m);
}

constexpr size_t ALIGN = 256;
size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Coefficients of the weight code: c_0 = 1, c_d = c_{d-1} ln2 / d in FP64,
// each rounded once to FP32; log2(e) rounded once to FP32.
QuantCoeffs make_qc() {
  QuantCoeffs q{};
  const double LN2 = 0.69314718055994530942;
  double d = 1.0;
  q.c[0] = 1.0f;
  for (int k = 1; k < 8; ++k) {
    d = d * LN2 / (double)k;
    q.c[k] = (float)d;
  }
  q.l2e = (float)1.4426950408889634;
  return q;
}

struct Layout {
  size_t trk, ts, gs, gd, tiles, frame_of, pv0, pv1, I0, I1, anc, lw, tp, ypad, hist, ghist, ring, ring_next, exo_next, keys_next,
      tile_ctr, parent, ds, rq, chunks, chunk_q, fsync,
      tmap, total;
  size_t rp_pv, rp_I, ck_pv, ck_I, ca_pv0, ca_pv1, ca_I0, ca_I1, lam_hist, lbar_hist, dlam, Dacc, grad, logz, seed,
      replay_bad;
  bool adjoint = false;
  int adj_slots = 0, adj_ckpts = 0;
  long long N_total = 0, ypad_total = 0, parent_total = 0, ghist_total = 0;
  int G_total = 0, n_tiles = 0, hist_total = 0, n_chunks = 0;
  int R = 5;
};

// Distance of the second log-weight buffer from the first: a multiple of
// 64 floats, so that both keep the 16-byte alignment the resampler's
// vector loads rely on.
long long lw_stride(long long N_total) { return (N_total + 63) / 64 * 64; }

// Padded frame geometry: a border of 2R+1 zero pixels, rows 16-byte
// aligned, and at least one TMA box in each dimension.
long long pad_pitch(int W, int R) {
  const long long p = ((long long)W + 2 * (2 * R + 1) + 3) / 4 * 4;
  return p < ROI_W ? ROI_W : p;
}
long long pad_rows(int H, int R) {
  const long long r = (long long)H + 2 * (2 * R + 1);
  return r < ROI_BOX_H ? ROI_BOX_H : r;
}

bool finite_nonneg(float v) { return std::isfinite(v) && v >= 0.0f; }

std::string validate(const pf_track_config* c, int n, int history) {
  if (!c) return "cfg is NULL";
  if (n < 1) return "n_tracks must be >= 1";
  if (history < 1) return "history must be >= 1";
  long long total = 0;
  for (int t = 0; t < n; ++t) {
    const pf_track_config& x = c[t];
    char b[160];
    auto bad = [&](const char* what) {
      std::snprintf(b, sizeof b, "track %d: %s", t, what);
      return std::string(b);
    };
    if (x.G < 1 || x.G > MAX_G) return bad("G must be in [1, 1024]");
    if (x.Np < 1 || x.Np > (1 << 20)) return bad("Np must be in [1, 2^20]");
    if (x.H < 1 || x.W < 1 || x.H > 16384 || x.W > 16384) return bad("H and W must be in [1, 16384]");
    if (x.patch_radius < 1 || x.patch_radius > 7) return bad("patch_radius must be in [1, 7]");
    if (x.patch_radius != c[0].patch_radius) return bad("all tracks must share patch_radius");
    if (x.mode != PF_RNA && x.mode != PF_ARNA) return bad("mode must be PF_RNA or PF_ARNA");
    if (x.init_kind < PF_INIT_POINT || x.init_kind > PF_INIT_USER) return bad("unknown init_kind");
    if (!(std::isfinite(x.sigma_psf) && x.sigma_psf > 0.0f)) return bad("sigma_psf must be > 0");
    if (!(std::isfinite(x.sigma_obs) && x.sigma_obs > 0.0f)) return bad("sigma_obs must be > 0");
    if (!std::isfinite(x.background)) return bad("background must be finite");
    if (!finite_nonneg(x.sigma_pos) || !finite_nonneg(x.sigma_v) || !finite_nonneg(x.sigma_I))
      return bad("process noise must be finite and >= 0");
    if (!(x.ex_ratio >= 0.0f && x.ex_ratio <= 1.0f)) return bad("ex_ratio must be in [0, 1]");
    if (!std::isfinite(x.pe_eff_cutoff)) return bad("pe_eff_cutoff must be finite");
    if (x.track_id >= (1u << 24)) return bad("track_id must be < 2^24");
    if (x.obs_model != PF_OBS_PATCH && x.obs_model != PF_OBS_FRAME) return bad("obs_model must be PF_OBS_PATCH or PF_OBS_FRAME");
    if (x.resample_rule != PF_RESAMPLE_ALWAYS && x.resample_rule != PF_RESAMPLE_ESS)
      return bad("resample_rule must be PF_RESAMPLE_ALWAYS or PF_RESAMPLE_ESS");
    if (!(x.ess_fraction >= 0.0f && x.ess_fraction <= 1.0f)) return bad("ess_fraction must be in [0, 1]");
    if (x.send_rule != PF_SEND_SYSTEMATIC && x.send_rule != PF_SEND_KEYED)
      return bad("send_rule must be PF_SEND_SYSTEMATIC or PF_SEND_KEYED");
    if (x.topology != PF_TOPO_RING && x.topology != PF_TOPO_NODE_RING && x.topology != PF_TOPO_HYPERCUBE)
      return bad("topology must be PF_TOPO_RING, PF_TOPO_NODE_RING or PF_TOPO_HYPERCUBE");
    if (x.topology == PF_TOPO_NODE_RING && x.node_groups < 1) return bad("node_groups must be >= 1");
    for (int d = 0; d < 5; ++d)
      if (!std::isfinite(x.init_state[d]) || !std::isfinite(x.init_lo[d]) || !std::isfinite(x.init_hi[d]))
        return bad("init_state / init_lo / init_hi must be finite");
    if (!finite_nonneg(x.init_radius)) return bad("init_radius must be finite and >= 0");
    total += (long long)x.G * x.Np;
  }
  if (total >= (1ll << 31)) return "total particles must be < 2^31";
  return "";
}

// Checkpoint spacing of pf_backward for T steps: ceil(sqrt(T)).
int adjoint_segment(int T) {
  int C = 1;
  while (C * C < T) ++C;
  return C;
}

Layout plan(const pf_track_config* c, int n, int history) {
  Layout L{};
  L.R = c[0].patch_radius;
  for (int t = 0; t < n; ++t) {
    const long long Nt = (long long)c[t].G * c[t].Np;
    L.N_total += Nt;
    L.G_total += c[t].G;
    L.n_tiles += c[t].G * ((c[t].Np + K1_TILE - 1) / K1_TILE);
    L.n_chunks += c[t].G * ((c[t].Np + RS_CHUNK - 1) / RS_CHUNK);
    L.ypad_total += pad_pitch(c[t].W, L.R) * pad_rows(c[t].H, L.R);
    if (c[t].record_ancestors) L.parent_total += Nt * history;
    L.hist_total += history;
    L.ghist_total += (long long)history * c[t].G;
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.ds = take(sizeof(DevState));
  L.tmap = take(sizeof(CUtensorMap) * n);
  L.trk = take(sizeof(TrackParams) * n);
  L.ts = take(sizeof(TrackState) * n);
  L.gs = take(sizeof(GroupState) * L.G_total);
  L.gd = take(sizeof(GroupDesc) * L.G_total);
  L.ring = take(sizeof(int) * L.G_total);
  L.ring_next = take(sizeof(int) * 2 * (size_t)L.G_total);
  L.exo_next = take(sizeof(uint32_t) * 2 * (size_t)L.G_total);
  L.keys_next = take(sizeof(uint4) * 2 * (size_t)L.G_total);
  L.tile_ctr = take(sizeof(int));
  L.rq = take(sizeof(unsigned int) * 4 * (size_t)L.n_chunks);
  L.chunks = take(sizeof(int4) * (size_t)L.n_chunks);
  L.chunk_q = take(4 * sizeof(unsigned long long) * (size_t)L.n_chunks);
  L.fsync = take(sizeof(unsigned int) * (size_t)FusedSync{L.G_total}.count());
  L.tiles = take(sizeof(int4) * L.n_tiles);
  L.frame_of = take(sizeof(int) * (size_t)n);
  L.pv0 = take(sizeof(float4) * L.N_total);
  L.pv1 = take(sizeof(float4) * L.N_total);
  L.I0 = take(sizeof(float) * L.N_total);
  L.I1 = take(sizeof(float) * L.N_total);
  L.anc = take(2 * sizeof(uint32_t) * L.N_total);  // by step parity
  L.lw = take(sizeof(float) * (size_t)lw_stride(L.N_total) * 2);
  L.tp = take(sizeof(float) * 8 * (size_t)L.n_tiles);
  L.ypad = take(sizeof(float) * (size_t)L.ypad_total);
  L.hist = take(sizeof(HistRec) * (size_t)L.hist_total);
  L.ghist = take(sizeof(GroupHist) * (size_t)L.ghist_total);
  L.parent = take(sizeof(uint32_t) * (size_t)(L.parent_total > 0 ? L.parent_total : 1));
  // pf_backward: every track must record its ancestry
  L.adjoint = true;
  for (int t = 0; t < n; ++t) L.adjoint = L.adjoint && c[t].record_ancestors;
  if (L.adjoint) {
    const int C = adjoint_segment(history);
    L.adj_slots = C < 2 ? 2 : C;
    L.adj_ckpts = (history + C - 1) / C + 1;
    L.rp_pv = take(sizeof(float4) * (size_t)L.N_total * L.adj_slots);
    L.rp_I = take(sizeof(float) * (size_t)L.N_total * L.adj_slots);
    L.ck_pv = take(sizeof(float4) * (size_t)L.N_total * L.adj_ckpts);
    L.ck_I = take(sizeof(float) * (size_t)L.N_total * L.adj_ckpts);
    L.ca_pv0 = take(sizeof(float4) * (size_t)L.N_total);
    L.ca_pv1 = take(sizeof(float4) * (size_t)L.N_total);
    L.ca_I0 = take(sizeof(float) * (size_t)L.N_total);
    L.ca_I1 = take(sizeof(float) * (size_t)L.N_total);
    L.lam_hist = take(sizeof(double) * (size_t)history * L.G_total);
    L.lbar_hist = take(sizeof(double) * (size_t)history * L.G_total);
    L.dlam = take(sizeof(double) * (size_t)L.G_total);
    L.Dacc = take(sizeof(double) * (size_t)L.G_total);
    L.grad = take(sizeof(double) * 5 * (size_t)n);
    L.logz = take(sizeof(double) * (size_t)n);
    L.seed = take(sizeof(float) * (size_t)n);
    L.replay_bad = take(sizeof(int));
  }
  L.total = o;
  return L;
}

int num_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

int resample_cluster(int Np, bool single_track) {
  if (!single_track) return 1;
  int c = (Np + RS_SUB - 1) / RS_SUB;
  return c < 1 ? 1 : (c > 8 ? 8 : c);
}

pf_status check_device(pf_handle* h) {
  DevState ds{};
  cudaError_t e = cudaMemcpy(&ds, h->ds, sizeof ds, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "reading the device error word");
  if (ds.err) {
    char b[200];
    std::snprintf(b, sizeof b, "kernel reported error bits 0x%x (info %u %u %u)", ds.err, ds.err_info[0],
                  ds.err_info[1], ds.err_info[2]);
    h->failed = 1;
    return fail(h, (ds.err & ERR_TIMEOUT) ? PF_ERR_TIMEOUT : PF_ERR_DEVICE, b);
  }
  return PF_OK;
}

// Records an event before (begin = true) or after a kernel when profiling.
cudaError_t mark(pf_handle* h, int kernel, cudaStream_t s) {
  if (!h->prof) return cudaSuccess;
  cudaEvent_t e;
  cudaError_t r = cudaEventCreate(&e);
  if (r != cudaSuccess) return r;
  h->ev[kernel].push_back(e);
  return cudaEventRecord(e, s);
}

// y = z - b into the padded frames, up to MAX_FRAMES_PER_LAUNCH tracks per
// launch.  frames: n_tracks device pointers.
// Blocks per frame of the frame preparation: enough for about sixteen
// 256-thread blocks per SM over the launch, each looping over rows, so that
// a batch of many small frames does not pay a block's start-up per row.
int prep_blocks(const pf_handle* h, int n_frames, int maxH) {
  const long long want = (16LL * h->sms + n_frames - 1) / n_frames;
  const int cap = maxH > 4096 ? 4096 : maxH;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

// Tracks of one launch given the same frame (pointer, size and background)
// share one padded copy, prepared once (several objects tracked in one
// sequence); frame_of tells the propagate kernel which copy each reads.
cudaError_t prep_frames(pf_handle* h, const float* const* frames, cudaStream_t s, bool share = true) {
  for (int t0 = 0; t0 < h->n_tracks; t0 += MAX_FRAMES_PER_LAUNCH) {
    const int nt = h->n_tracks - t0 < MAX_FRAMES_PER_LAUNCH ? h->n_tracks - t0 : MAX_FRAMES_PER_LAUNCH;
    FrameArgs a;
    a.trk = h->trk;
    a.ypad = h->ypad;
    a.frame_of = h->frame_of;
    a.t0 = t0;
    a.nt = nt;
    a.R = h->R;
    int maxH = 1, n_rep = 0;
    std::unordered_map<const float*, int> first;
    for (int i = 0; i < nt; ++i) {
      const int t = t0 + i;
      a.frames[i] = frames[t];
      const pf_track_config& c = h->cfg[t];
      auto it = first.find(frames[t]);
      const bool same = it != first.end() && h->cfg[it->second].H == c.H && h->cfg[it->second].W == c.W &&
                        h->tp[it->second].bg == h->tp[t].bg;
      if (same && share) {
        a.share[i] = it->second;
      } else {
        first[frames[t]] = t;
        a.share[i] = t;
        a.rep[n_rep++] = (short)i;
        if (c.H > maxH) maxH = c.H;
      }
    }
    cudaError_t e = launch_frame_prep(a, n_rep, prep_blocks(h, n_rep, maxH), h->pdl, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

GlobalArgs global_args(const pf_handle* h, int finalize);

// Wait for the handle's last stream, after completing the last step's
// estimate, log Z and history (k_finish) if no later step has done it.
pf_status sync(pf_handle* h) {
  if (h->finish_pending) {
    const cudaError_t ef = launch_finish(global_args(h, 1), h->n_tracks, h->last_stream);
    if (ef != cudaSuccess) return cuda_fail(h, ef, "k_finish");
    h->finish_pending = false;
  }
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
  return check_device(h);
}

K1Args k1_args(const pf_handle* h) {
  K1Args a{};
  a.trk = h->trk;
  a.tiles = h->tiles;
  a.n_tiles = h->n_tiles;
  a.grp = h->gs;
  a.ts = h->ts;
  a.ds = h->ds;
  a.pv0 = h->pv[0];
  a.pv1 = h->pv[1];
  a.I0 = h->In[0];
  a.I1 = h->In[1];
  a.anc = h->anc;
  a.anc_stride = h->N_total;
  a.parent = h->parent;
  a.history = h->history;
  a.lw = h->lw;
  a.lw1 = h->carry_any ? h->lw + lw_stride(h->N_total) : h->lw;
  a.tile_part = h->tile_part;
  a.ypad = h->ypad;
  a.tmaps = h->tmaps;
  a.ring_next = h->ring_next;
  a.ring_stride = h->G_total;
  a.ring = h->ring;
  a.exo_next = h->exo_next;
  a.hist = h->hist;
  a.ghist = h->ghist;
  a.tile_ctr = h->tile_ctr;
  a.n_ring_blocks = h->n_ring_blocks;
  a.n_tracks = h->n_tracks;
  a.p0 = h->tp[0];
  a.raw_frame = 0;
  a.zraw = nullptr;
  a.test_withhold_copy = h->test_withhold_copy ? 1 : 0;
  a.variants = h->variants ? 1 : 0;
  a.keys_next = h->keys_next;
  a.frame_of = h->frame_of;
  a.n_chunks = h->n_chunks;
  a.chunks = h->chunks;
  a.gd = h->gd;
  a.chunk_q = h->chunk_q;
  a.sync = h->fsync;
  a.rq = h->rq;
  a.qc = h->qc;
  return a;
}

// A single-track step reads the caller's frame directly (no frame
// preparation kernel) when a TMA descriptor can describe it: the driver
// entry point is available, the frame starts on 16 bytes, its rows are a
// multiple of 16 bytes and it holds at least one staging box.  Sets the
// descriptor in `a` and returns true, else leaves `a` unchanged.
bool raw_frame_map(const pf_handle* h, const float* frame, K1Args* a) {
  if (h->n_tracks != 1 || !h->encode || !frame) return false;
  const pf_track_config& c = h->cfg[0];
  if (((uintptr_t)frame & 15) != 0 || (c.W % 4) != 0 || c.W < ROI_W || c.H < ROI_BOX_H) return false;
  cuuint64_t dims[2] = {(cuuint64_t)c.W, (cuuint64_t)c.H};
  cuuint64_t strides[1] = {(cuuint64_t)c.W * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)ROI_W, (cuuint32_t)ROI_BOX_H};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMap m;
  const CUresult r = ((PFN_cuTensorMapEncodeTiled_v12000)h->encode)(
      &m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)frame, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  a->raw_frame = 1;
  a->zraw = frame;
  a->zmap = m;
  return true;
}

GlobalArgs global_args(const pf_handle* h, int finalize) {
  return GlobalArgs{h->trk, h->ts, h->gs, h->ring, h->ring_next, h->G_total, h->exo_next, h->hist, h->ghist, h->history,
                    finalize, h->ds};
}

// fuse = 1: the resampler also runs each track's global step (the last
// group of the track to finish); 0: resampling only (autotuner candidates).
ResampleArgs resample_args(const pf_handle* h, int fuse) {
  ResampleArgs ra{h->gd,  h->gs,  h->tile_part, h->lw, h->carry_any ? h->lw + lw_stride(h->N_total) : nullptr,
                  h->anc, h->N_total, nullptr, nullptr, 0, h->qc, h->ds};
  // one track: the global step on an extra cluster of the launch, so that the
  // group that reports last goes straight on to its own merge
  ra.fuse_global = (fuse == 1 && h->n_tracks == 1 && h->global_cta) ? 2 : fuse;
  ra.n_groups = h->G_total;
  ra.lean = h->carry_any ? 0 : 1;  // no group resamples by Alg. 1's test
  ra.max_np = 1;
  for (int t = 0; t < h->n_tracks; ++t) ra.max_np = h->cfg[t].Np > ra.max_np ? h->cfg[t].Np : ra.max_np;
  ra.tile_ctr = h->tile_ctr;
  ra.glob = global_args(h, 1);
  return ra;
}

}  // namespace

namespace pf {
QuantCoeffs resample_coeffs() { return make_qc(); }
int resample_cluster_size(int Np) { return resample_cluster(Np, true); }
void set_handleless_error(const char* msg) { g_err = msg; }
}  // namespace pf

extern "C" {

int32_t pf_abi_version(void) { return PF_ABI_VERSION; }

pf_status pf_query_workspace(const pf_track_config* cfg, int32_t n_tracks, int32_t history, size_t* bytes) {
  if (!bytes) return fail(nullptr, PF_ERR_ARG, "bytes is NULL");
  const std::string v = validate(cfg, n_tracks, history);
  if (!v.empty()) return fail(nullptr, PF_ERR_ARG, v);
  *bytes = plan(cfg, n_tracks, history).total;
  return PF_OK;
}

pf_status pf_init(const pf_track_config* cfg, int32_t n_tracks, int32_t history, void* workspace, size_t bytes,
                  const float* user_state, void* stream, pf_handle** out) {
  NvtxRange nvtx_range("pf_init");
  if (!out) return fail(nullptr, PF_ERR_ARG, "out is NULL");
  *out = nullptr;
  const std::string v = validate(cfg, n_tracks, history);
  if (!v.empty()) return fail(nullptr, PF_ERR_ARG, v);
  if (!workspace) return fail(nullptr, PF_ERR_ARG, "workspace is NULL");
  if ((uintptr_t)workspace % ALIGN) return fail(nullptr, PF_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  const Layout L = plan(cfg, n_tracks, history);
  if (bytes < L.total) return fail(nullptr, PF_ERR_WORKSPACE, "workspace too small");
  bool need_user = false;
  for (int t = 0; t < n_tracks; ++t) need_user |= cfg[t].init_kind == PF_INIT_USER;
  if (need_user && !user_state) return fail(nullptr, PF_ERR_ARG, "PF_INIT_USER needs user_state_dev");

  pf_handle* h = new pf_handle();
  h->n_tracks = n_tracks;
  h->history = history;
  h->R = L.R;
  h->cfg.assign(cfg, cfg + n_tracks);
  h->N_total = L.N_total;
  h->G_total = L.G_total;
  h->n_tiles = L.n_tiles;
  h->qc = make_qc();
  {
    const char* v = std::getenv("PFARNA_PDL");  // "0": plain stream serialisation between step kernels
    h->pdl = !(v && v[0] == '0');
    const char* tw = std::getenv("PFARNA_TEST_WITHHOLD_COPY");
    h->test_withhold_copy = tw && tw[0] == '1';
  }
  h->last_stream = (cudaStream_t)stream;
  char* w = (char*)workspace;
  h->ds = (DevState*)(w + L.ds);
  h->trk = (TrackParams*)(w + L.trk);
  h->ts = (TrackState*)(w + L.ts);
  h->gs = (GroupState*)(w + L.gs);
  h->gd = (GroupDesc*)(w + L.gd);
  h->ring = (int*)(w + L.ring);
  h->ring_next = (int*)(w + L.ring_next);
  h->exo_next = (uint32_t*)(w + L.exo_next);
  h->keys_next = (uint4*)(w + L.keys_next);
  h->tile_ctr = (int*)(w + L.tile_ctr);
  h->rq = (unsigned int*)(w + L.rq);
  h->chunks = (int4*)(w + L.chunks);
  h->n_chunks = L.n_chunks;
  h->chunk_q = (unsigned long long*)(w + L.chunk_q);
  h->fsync = (unsigned int*)(w + L.fsync);
  h->tiles = (int4*)(w + L.tiles);
  h->frame_of = (int*)(w + L.frame_of);
  h->pv[0] = (float4*)(w + L.pv0);
  h->pv[1] = (float4*)(w + L.pv1);
  h->In[0] = (float*)(w + L.I0);
  h->In[1] = (float*)(w + L.I1);
  h->anc = (uint32_t*)(w + L.anc);
  h->lw = (float*)(w + L.lw);
  h->tile_part = (float*)(w + L.tp);
  h->ypad = (float*)(w + L.ypad);
  h->hist = (HistRec*)(w + L.hist);
  h->ghist = (GroupHist*)(w + L.ghist);
  h->parent = (uint32_t*)(w + L.parent);
  h->tmaps = (CUtensorMap*)(w + L.tmap);
  if (L.adjoint) {
    h->adjoint = true;
    h->adj_slots = L.adj_slots;
    h->adj_ckpts = L.adj_ckpts;
    h->rp_pv = (float4*)(w + L.rp_pv);
    h->rp_I = (float*)(w + L.rp_I);
    h->ck_pv = (float4*)(w + L.ck_pv);
    h->ck_I = (float*)(w + L.ck_I);
    h->ca_pv[0] = (float4*)(w + L.ca_pv0);
    h->ca_pv[1] = (float4*)(w + L.ca_pv1);
    h->ca_I[0] = (float*)(w + L.ca_I0);
    h->ca_I[1] = (float*)(w + L.ca_I1);
    h->lam_hist = (double*)(w + L.lam_hist);
    h->lbar_hist = (double*)(w + L.lbar_hist);
    h->dlam = (double*)(w + L.dlam);
    h->Dacc = (double*)(w + L.Dacc);
    h->grad = (double*)(w + L.grad);
    h->logz_rp = (double*)(w + L.logz);
    h->seed = (float*)(w + L.seed);
    h->replay_bad = (int*)(w + L.replay_bad);
  }

  // host tables
  std::vector<TrackParams> tp(n_tracks);
  std::vector<GroupDesc> gd;
  std::vector<int4> tiles;
  std::vector<int4> chunks;  // fused step: (track, global group, first slot, items)
  gd.reserve(L.G_total);
  tiles.reserve(L.n_tiles);
  chunks.reserve(L.n_chunks);
  long long part = 0, ypo = 0, paro = 0, gho = 0;
  int gro = 0, tio = 0, ho = 0;
  for (int t = 0; t < n_tracks; ++t) {
    const pf_track_config& c = cfg[t];
    TrackParams& P = tp[t];
    std::memset(&P, 0, sizeof P);
    P.G = c.G; P.Np = c.Np; P.H = c.H; P.W = c.W;
    P.mode = c.mode; P.init_kind = c.init_kind;
    P.spsf = c.sigma_psf; P.bg = c.background; P.sobs = c.sigma_obs;
    P.spos = c.sigma_pos; P.sv = c.sigma_v; P.sI = c.sigma_I;
    P.ex_ratio = c.ex_ratio; P.cutoff = c.pe_eff_cutoff;
    P.c_psf = (float)(1.4426950408889634 / (2.0 * (double)c.sigma_psf * (double)c.sigma_psf));
    P.inv2so2 = (float)(1.0 / (2.0 * (double)c.sigma_obs * (double)c.sigma_obs));
    P.kappa = (float)std::exp2(-2.0 * (double)P.c_psf);
    P.key0 = (uint32_t)c.seed;
    P.key1 = (uint32_t)(c.seed >> 32);
    for (int r = 0; r < 10; ++r) {
      P.rk[2 * r] = P.key0 + (uint32_t)r * 0x9E3779B9u;
      P.rk[2 * r + 1] = P.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    P.tag = c.track_id << 8;
    P.record = c.record_ancestors ? 1 : 0;
    P.obs_model = c.obs_model;
    P.resample_rule = c.resample_rule;
    P.ess_t = (uint32_t)std::floor((double)c.ess_fraction * 65536.0 + 0.5);
    P.send_rule = c.send_rule;
    P.topology = c.topology;
    P.node_groups = c.node_groups < 1 ? 1 : c.node_groups;
    P.hyper_dims = 0;
    while ((1 << P.hyper_dims) < c.G) ++P.hyper_dims;
    P.perm_bits = 0;
    while ((1 << P.perm_bits) < c.Np) ++P.perm_bits;
    P.part_off = part;
    P.group_off = gro;
    P.tile_off = tio;
    P.tiles_per_group = (c.Np + K1_TILE - 1) / K1_TILE;
    P.m_Np = fastdiv_magic((uint32_t)c.Np);
    P.pitch = (int)pad_pitch(c.W, L.R);
    P.ypad_off = ypo;
    P.hist_off = ho;
    P.ghist_off = gho;
    P.parent_off = paro;
    for (int d = 0; d < 5; ++d) {
      P.init_state[d] = c.init_state[d];
      P.init_lo[d] = c.init_lo[d];
      P.init_hi[d] = c.init_hi[d];
    }
    P.init_radius = c.init_radius;
    for (int g = 0; g < c.G; ++g) {
      GroupDesc D{};
      D.base = part + (long long)g * c.Np;
      D.Np = c.Np;
      D.track = t;
      D.g = g;
      D.tile_begin = (int)tiles.size();
      for (int j0 = 0; j0 < c.Np; j0 += K1_TILE)
        tiles.push_back(make_int4(t, g, j0, c.Np - j0 < K1_TILE ? c.Np - j0 : K1_TILE));
      D.tile_count = (int)tiles.size() - D.tile_begin;
      D.chunk_begin = (int)chunks.size();
      for (int j0 = 0; j0 < c.Np; j0 += RS_CHUNK)
        chunks.push_back(make_int4(t, gro + g, j0, c.Np - j0 < RS_CHUNK ? c.Np - j0 : RS_CHUNK));
      D.chunk_count = (int)chunks.size() - D.chunk_begin;
      gd.push_back(D);
    }
    const long long Nt = (long long)c.G * c.Np;
    part += Nt;
    gro += c.G;
    tio += c.G * P.tiles_per_group;
    ypo += (long long)P.pitch * pad_rows(c.H, L.R);
    ho += history;
    gho += (long long)history * c.G;
    if (c.record_ancestors) paro += Nt * history;
  }
  h->tp = tp;
  cudaStream_t s = (cudaStream_t)stream;

  // One TMA descriptor per track over its padded frame (boxes of ROI_W x
  // ROI_BOX_H floats).  If the driver cannot encode them, the propagate
  // kernel reads every frame through L1 instead.
  std::vector<CUtensorMap> maps(n_tracks);
  {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    bool ok = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                  cudaSuccess && q == cudaDriverEntryPointSuccess && fn != nullptr;
    for (int t = 0; ok && t < n_tracks; ++t) {
      const TrackParams& P = tp[t];
      cuuint64_t dims[2] = {(cuuint64_t)P.pitch, (cuuint64_t)pad_rows(P.H, L.R)};
      cuuint64_t strides[1] = {(cuuint64_t)P.pitch * sizeof(float)};
      cuuint32_t box[2] = {(cuuint32_t)ROI_W, (cuuint32_t)ROI_BOX_H};
      cuuint32_t estr[2] = {1, 1};
      CUresult r = ((PFN_cuTensorMapEncodeTiled_v12000)fn)(
          &maps[t], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)(h->ypad + P.ypad_off), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      ok = (r == CUDA_SUCCESS);
    }
    if (!ok) h->tmaps = nullptr;
    if (ok) h->encode = fn;
  }
  std::vector<int> ident(n_tracks);  // every track reads its own padded frame until a step shares one
  for (int t = 0; t < n_tracks; ++t) ident[t] = t;
  cudaError_t e;
  if ((e = cudaMemsetAsync(w, 0, L.total, s)) != cudaSuccess) { pf_destroy(h); return cuda_fail(nullptr, e, "cudaMemsetAsync"); }
  if ((e = cudaMemcpyAsync(h->trk, tp.data(), sizeof(TrackParams) * n_tracks, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(h->gd, gd.data(), sizeof(GroupDesc) * gd.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(h->tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(h->chunks, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(h->frame_of, ident.data(), sizeof(int) * ident.size(), cudaMemcpyHostToDevice, s)) ||
      (h->tmaps && (e = cudaMemcpyAsync(h->tmaps, maps.data(), sizeof(CUtensorMap) * n_tracks,
                                        cudaMemcpyHostToDevice, s)))) {
    pf_destroy(h);
    return cuda_fail(nullptr, e, "uploading track tables");
  }
  // the staging copies above read pageable host memory, so they complete
  // (from the host's point of view) before returning; the vectors may go.

  const int sms = num_sms();
  h->sms = sms;
  h->ws = w;
  h->ws_total = L.total;
  h->tmap_off = L.tmap;
  h->tmap_bytes = sizeof(CUtensorMap) * (size_t)n_tracks;
  {
    // FNV-1a over the configurations and the history length
    unsigned long long sig = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
      for (size_t i = 0; i < n; ++i) sig = (sig ^ ((const unsigned char*)p)[i]) * 1099511628211ull;
    };
    mix(cfg, sizeof(pf_track_config) * (size_t)n_tracks);
    mix(&history, sizeof history);
    mix(&L.total, sizeof L.total);
    h->cfg_sig = sig;
  }
  int occ = 1;
  if ((e = k1_occupancy(h->R, &occ)) != cudaSuccess) { pf_destroy(h); return cuda_fail(nullptr, e, "occupancy"); }
  h->k1_occ = occ > 0 ? occ : 1;
  const long long want = (long long)sms * (occ > 0 ? occ : 1);
  h->k1_grid = (int)(h->n_tiles < want ? h->n_tiles : want);
  int n_arna = 0;
  for (int t = 0; t < n_tracks; ++t) n_arna += (cfg[t].mode == PF_ARNA && cfg[t].G > 1 && cfg[t].G <= RING_SMEM_G);
  (void)n_arna;
  h->n_ring_blocks = n_tracks < 16 ? n_tracks : 16;
  {
    // PFARNA_FUSED=1: the one-launch (fused) step instead of propagate, then
    // resample; measured slower on the tracking and batched workloads, so not
    // the default
    const char* fz = std::getenv("PFARNA_FUSED");
    h->fused = fz && std::atoi(fz) == 1;
    const char* gc = std::getenv("PFARNA_GLOBAL_CTA");
    h->global_cta = !(gc && std::atoi(gc) == 0);
    int focc = 1;
    if ((e = fused_occupancy(h->R, &focc)) != cudaSuccess) { pf_destroy(h); return cuda_fail(nullptr, e, "occupancy"); }
    if (focc < 1) focc = 1;
    const int n_tasks = L.n_tiles + 2 * L.n_chunks;
    const long long fw = (long long)sms * focc;
    h->fused_grid = (int)(n_tasks < fw ? n_tasks : fw);
  }
  for (int t = 0; t < n_tracks; ++t) {
    h->max_G = cfg[t].G > h->max_G ? cfg[t].G : h->max_G;
    if (cfg[t].resample_rule == PF_RESAMPLE_ESS) h->carry_any = true;
    if (cfg[t].resample_rule == PF_RESAMPLE_ESS || cfg[t].send_rule == PF_SEND_KEYED) h->variants = true;
  }
  {
    // resampler shape: small CTAs (eight per SM) when every group fits one
    // of their sub-chunks; clusters sized to the largest group, as long as
    // the launch stays within about two waves of two CTAs per SM
    int maxNp = 1;
    for (int t = 0; t < n_tracks; ++t) maxNp = cfg[t].Np > maxNp ? cfg[t].Np : maxNp;
    h->rs_threads = maxNp <= RS_THREADS_SMALL * RS_ITEMS ? RS_THREADS_SMALL : RS_THREADS;
    if (n_tracks == 1) {
      h->rs_cluster = resample_cluster(cfg[0].Np, true);
    } else {
      const int sub = h->rs_threads * RS_ITEMS;
      int c = (maxNp + sub - 1) / sub;
      c = c < 1 ? 1 : (c > 8 ? 8 : c);
      while (c > 1 && (long long)h->G_total * c > 4LL * h->sms) c >>= 1;
      h->rs_cluster = c;
    }
    const char* rt = std::getenv("PFARNA_RS_THREADS");  // "128" / "512": force the resampler's CTA size
    if (rt && std::atoi(rt) == RS_THREADS_SMALL) h->rs_threads = RS_THREADS_SMALL;
    if (rt && std::atoi(rt) == RS_THREADS) h->rs_threads = RS_THREADS;
  }

  InitArgs ia{h->trk, h->tiles, h->n_tiles, h->N_total, user_state, h->pv[1], h->In[1]};
  if ((e = launch_init(ia, h->k1_grid, s)) != cudaSuccess) { pf_destroy(h); return cuda_fail(nullptr, e, "k_init"); }
  if ((e = launch_global(global_args(h, 0), n_tracks, s)) != cudaSuccess) {
    pf_destroy(h);
    return cuda_fail(nullptr, e, "k_global");
  }
  *out = h;
  return PF_OK;
}

// The kernels of one step after frame preparation: the fused step, or
// propagate + weight, then resample with the global step as its tail.
// marks: record profiling events (not while a graph is being captured).
static cudaError_t launch_step_kernels(pf_handle* h, cudaStream_t s, bool marks, const K1Args* k1p = nullptr) {
  const K1Args k1 = k1p ? *k1p : k1_args(h);
  cudaError_t e;
  if (h->fused) {
    if (marks && (e = mark(h, PF_KERNEL_FUSED_STEP, s)) != cudaSuccess) return e;
    if ((e = launch_fused_step(k1, h->R, h->fused_grid + h->n_ring_blocks, h->pdl, s)) != cudaSuccess) return e;
    return marks ? mark(h, PF_KERNEL_FUSED_STEP, s) : cudaSuccess;
  }
  if (marks && (e = mark(h, PF_KERNEL_PROPAGATE_WEIGHT, s)) != cudaSuccess) return e;
  if ((e = launch_propagate(k1, h->R, h->k1_grid + h->n_ring_blocks, h->pdl, s)) != cudaSuccess) return e;
  if (marks && (e = mark(h, PF_KERNEL_PROPAGATE_WEIGHT, s)) != cudaSuccess) return e;
  if (marks && (e = mark(h, PF_KERNEL_RESAMPLE, s)) != cudaSuccess) return e;
  if ((e = launch_resample(resample_args(h, 1), h->G_total, h->rs_cluster, h->pdl, s, h->rs_threads)) != cudaSuccess)
    return e;
  return marks ? mark(h, PF_KERNEL_RESAMPLE, s) : cudaSuccess;
}

pf_status pf_step(pf_handle* h, const float* const* frames, void* stream) {
  NvtxRange nvtx_range("pf_step");
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (h->failed) return fail(h, PF_ERR_STATE, "handle failed earlier: " + h->err);
  if (!frames) return fail(h, PF_ERR_ARG, "frames is NULL");
  for (int t = 0; t < h->n_tracks; ++t)
    if (!frames[t]) return fail(h, PF_ERR_ARG, "frame pointer of track " + std::to_string(t) + " is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  K1Args k1 = k1_args(h);
  if (h->variants || !raw_frame_map(h, frames[0], &k1)) {
    if ((e = mark(h, PF_KERNEL_FRAME_PREP, s)) != cudaSuccess) return cuda_fail(h, e, "profile event");
    if ((e = prep_frames(h, frames, s)) != cudaSuccess) return cuda_fail(h, e, "k_frame_prep");
    if ((e = mark(h, PF_KERNEL_FRAME_PREP, s)) != cudaSuccess) return cuda_fail(h, e, "profile event");
  }
  if ((e = launch_step_kernels(h, s, true, &k1)) != cudaSuccess) return cuda_fail(h, e, "step kernels");
  h->steps_run += 1;
  h->finish_pending = true;
  h->last_stream = s;
  return PF_OK;
}

// pf_step_host's staging: two slots (by step parity), each holding every
// track's frame at a 256-byte aligned offset.
static size_t staging_slot_bytes(const pf_handle* h, std::vector<size_t>* off) {
  size_t n = 0;
  for (int t = 0; t < h->n_tracks; ++t) {
    if (off) off->push_back(n);
    n += ((size_t)h->cfg[t].H * h->cfg[t].W * sizeof(float) + 255) & ~(size_t)255;
  }
  return n;
}

pf_status pf_host_staging_bytes(const pf_handle* h, size_t* bytes) {
  if (!h || !bytes) return fail(nullptr, PF_ERR_ARG, "handle or output is NULL");
  *bytes = 2 * staging_slot_bytes(h, nullptr);
  return PF_OK;
}

pf_status pf_step_host(pf_handle* h, const float* const* frames_host, void* staging_dev, size_t staging_bytes,
                       void* stream) {
  NvtxRange nvtx_range("pf_step_host");
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (h->failed) return fail(h, PF_ERR_STATE, "handle failed earlier: " + h->err);
  if (!frames_host) return fail(h, PF_ERR_ARG, "frames is NULL");
  for (int t = 0; t < h->n_tracks; ++t)
    if (!frames_host[t]) return fail(h, PF_ERR_ARG, "frame pointer of track " + std::to_string(t) + " is NULL");
  std::vector<size_t> off;
  const size_t slot_bytes = staging_slot_bytes(h, &off);
  if (!staging_dev || ((uintptr_t)staging_dev & 255) != 0)
    return fail(h, PF_ERR_ARG, "staging buffer is NULL or not 256-byte aligned");
  if (staging_bytes < 2 * slot_bytes) return fail(h, PF_ERR_ARG, "staging buffer is smaller than pf_host_staging_bytes");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!h->up_stream) {
    if ((e = cudaStreamCreateWithFlags(&h->up_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(h, e, "creating the upload stream");
    for (int i = 0; i < 2; ++i)
      if ((e = cudaEventCreateWithFlags(&h->up_copied[i], cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&h->up_used[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(h, e, "creating upload events");
  }
  const int slot = h->steps_run & 1;
  char* base = (char*)staging_dev + (size_t)slot * slot_bytes;
  // the step two back read this slot (an event never recorded waits for nothing)
  if ((e = cudaStreamWaitEvent(h->up_stream, h->up_used[slot], 0)) != cudaSuccess)
    return cuda_fail(h, e, "upload stream wait");
  std::vector<const float*> dev(h->n_tracks);
  std::unordered_map<const float*, int> first;  // a host frame given to several tracks is uploaded once
  for (int t = 0; t < h->n_tracks; ++t) {
    const size_t n = (size_t)h->cfg[t].H * h->cfg[t].W * sizeof(float);
    auto it = first.find(frames_host[t]);
    if (it != first.end() && (size_t)h->cfg[it->second].H * h->cfg[it->second].W * sizeof(float) == n) {
      dev[t] = dev[it->second];
      continue;
    }
    first.emplace(frames_host[t], t);
    dev[t] = reinterpret_cast<const float*>(base + off[t]);
    if ((e = cudaMemcpyAsync(base + off[t], frames_host[t], n, cudaMemcpyHostToDevice, h->up_stream)) != cudaSuccess)
      return cuda_fail(h, e, "frame upload");
  }
  if ((e = cudaEventRecord(h->up_copied[slot], h->up_stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(s, h->up_copied[slot], 0)) != cudaSuccess)
    return cuda_fail(h, e, "upload event");
  const pf_status st = pf_step(h, dev.data(), stream);
  if (st != PF_OK) return st;
  if ((e = cudaEventRecord(h->up_used[slot], s)) != cudaSuccess) return cuda_fail(h, e, "upload event");
  return PF_OK;
}

static cudaError_t launch_frames_table(pf_handle* h, const float* const* table, int T_table, cudaStream_t s) {
  int maxH = 1;
  for (int t = 0; t < h->n_tracks; ++t) maxH = h->cfg[t].H > maxH ? h->cfg[t].H : maxH;
  FrameTableArgs fa{h->trk, h->ypad, h->R, table, T_table, h->n_tracks, h->ts, h->ds, h->frame_of};
  return launch_frame_prep_table(fa, prep_blocks(h, h->n_tracks, maxH), h->pdl, s);
}

pf_status pf_step_table(pf_handle* h, const float* const* table_dev, int32_t T_table, void* stream) {
  NvtxRange nvtx_range("pf_step_table");
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (h->failed) return fail(h, PF_ERR_STATE, "handle failed earlier: " + h->err);
  if (!table_dev || T_table < 1) return fail(h, PF_ERR_ARG, "bad frame table");
  if (h->n_tracks > 65535) return fail(h, PF_ERR_ARG, "frame tables serve at most 65535 tracks");
  if (h->steps_run >= T_table) return fail(h, PF_ERR_STATE, "the frame table has no frame for this step");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = mark(h, PF_KERNEL_FRAME_PREP, s)) != cudaSuccess) return cuda_fail(h, e, "profile event");
  if ((e = launch_frames_table(h, table_dev, T_table, s)) != cudaSuccess) return cuda_fail(h, e, "k_frame_prep_table");
  if ((e = mark(h, PF_KERNEL_FRAME_PREP, s)) != cudaSuccess) return cuda_fail(h, e, "profile event");
  if ((e = launch_step_kernels(h, s, true)) != cudaSuccess) return cuda_fail(h, e, "step kernels");
  h->steps_run += 1;
  h->finish_pending = true;
  h->last_stream = s;
  return PF_OK;
}

pf_status pf_graph_step(pf_handle* h, const float* const* table_dev, int32_t T_table, void* stream) {
  NvtxRange nvtx_range("pf_graph_step");
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (h->failed) return fail(h, PF_ERR_STATE, "handle failed earlier: " + h->err);
  if (!table_dev || T_table < 1) return fail(h, PF_ERR_ARG, "bad frame table");
  if (h->n_tracks > 65535) return fail(h, PF_ERR_ARG, "frame tables serve at most 65535 tracks");
  if (h->steps_run >= T_table) return fail(h, PF_ERR_STATE, "the frame table has no frame for this step");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!h->graph || h->graph_table != (const void*)table_dev || h->graph_T != T_table) {
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
    // capture the parameter-free step once; its kernels read the step index
    // and frame pointers on the device
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(h, e, "capture stream");
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = launch_frames_table(h, table_dev, T_table, cs);
      cudaError_t e2 = e1 == cudaSuccess ? launch_step_kernels(h, cs, false) : e1;
      e = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(h, e, "capturing the step graph");
    h->graph_table = table_dev;
    h->graph_T = T_table;
  }
  if ((e = cudaGraphLaunch(h->graph, s)) != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
  h->steps_run += 1;
  h->finish_pending = true;
  h->last_stream = s;
  return PF_OK;
}

// Autotuner results by problem shape (tracks, particles, groups, largest
// group, SMs): propagate grid and resampler cluster size.
static std::mutex g_tune_mutex;
static std::map<std::tuple<int, long long, int, int, int>, std::tuple<int, int, int>> g_tune_cache;

pf_status pf_autotune(pf_handle* h, const float* const* frames, int32_t* k1_grid_out, int32_t* cluster_out,
                      void* stream) {
  NvtxRange nvtx_range("pf_autotune");
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (h->failed) return fail(h, PF_ERR_STATE, "handle failed earlier: " + h->err);
  if (!frames) return fail(h, PF_ERR_ARG, "frames is NULL");
  for (int t = 0; t < h->n_tracks; ++t)
    if (!frames[t]) return fail(h, PF_ERR_ARG, "NULL frame pointer");
  cudaStream_t s = (cudaStream_t)stream;
  int maxNp = 1;
  for (int t = 0; t < h->n_tracks; ++t) maxNp = h->cfg[t].Np > maxNp ? h->cfg[t].Np : maxNp;
  const auto key = std::make_tuple(h->n_tracks, h->N_total, h->G_total, maxNp, h->sms);
  cudaError_t e;
  if ((e = prep_frames(h, frames, s)) != cudaSuccess) return cuda_fail(h, e, "k_frame_prep");
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      h->k1_grid = std::get<0>(it->second);
      h->rs_cluster = std::get<1>(it->second);
      h->rs_threads = std::get<2>(it->second);
      cached = true;
    }
  }
  if (!cached) {
    // Within a step the propagate kernel is idempotent until a resampler
    // replaces the ancestors it reads, and the resampler is idempotent until
    // the global step advances the step: the propagate candidates are timed
    // first, then the resampler's, on live data.
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_it = [&](auto&& launch, float& ms) -> cudaError_t {
      cudaError_t r = cudaEventRecord(e0, s);
      if (r == cudaSuccess) r = launch();
      if (r == cudaSuccess) r = cudaEventRecord(e1, s);
      if (r == cudaSuccess) r = cudaEventSynchronize(e1);
      if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
      return r;
    };
    const K1Args k1 = k1_args(h);
    int best_grid = h->k1_grid;
    float best = 1e30f;
    for (int b = 1; b <= h->k1_occ; ++b) {
      const long long cand = (long long)h->sms * b;
      const int grid = (int)(cand < h->n_tiles ? cand : h->n_tiles);
      float ms = 0.0f;
      for (int rep = 0; rep < 2; ++rep)  // the first run also warms caches
        if ((e = time_it(
                 [&] {
                   cudaError_t r = cudaMemsetAsync(h->tile_ctr, 0, sizeof(int), s);
                   return r != cudaSuccess ? r : launch_propagate(k1, h->R, grid + h->n_ring_blocks, false, s);
                 },
                 ms)) != cudaSuccess)
          break;
      if (e != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        best_grid = grid;
      }
      if (grid == h->n_tiles) break;
    }
    int best_c = h->rs_cluster, best_t = h->rs_threads;
    best = 1e30f;
    for (int nt : {RS_THREADS, RS_THREADS_SMALL})
      for (int c = 1; c <= 8 && e == cudaSuccess; c *= 2) {
        const ResampleArgs ra = resample_args(h, 0);
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep)
          if ((e = time_it([&] { return launch_resample(ra, h->G_total, c, false, s, nt); }, ms)) != cudaSuccess) break;
        if (e != cudaSuccess) break;
        if (ms < best) {
          best = ms;
          best_c = c;
          best_t = nt;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
    h->k1_grid = best_grid;
    h->rs_cluster = best_c;
    h->rs_threads = best_t;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = std::make_tuple(best_grid, best_c, best_t);
  }
  // Complete the step with the chosen shapes.  When candidates were timed,
  // the propagate candidates (which run first) have left this step's states
  // and weights, and the resampler candidates have replaced the ancestors
  // the propagate kernel reads, so only the resampler runs again, now with
  // the global step.
  e = cached ? launch_step_kernels(h, s, false)
             : launch_resample(resample_args(h, 1), h->G_total, h->rs_cluster, false, s, h->rs_threads);
  if (e != cudaSuccess) return cuda_fail(h, e, "step kernels");
  h->steps_run += 1;
  h->finish_pending = true;
  h->last_stream = s;
  if (h->graph) {  // a captured step holds the old shapes
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (k1_grid_out) *k1_grid_out = h->k1_grid;
  if (cluster_out) *cluster_out = h->rs_cluster;
  return PF_OK;
}

pf_status pf_estimate(pf_handle* h, float* xhat, double* logZ) {
  NvtxRange nvtx_range("pf_estimate");
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (h->steps_run == 0) return fail(h, PF_ERR_STATE, "no step has run");
  pf_status st = sync(h);
  if (st != PF_OK) return st;
  std::vector<TrackState> ts(h->n_tracks);
  cudaError_t e = cudaMemcpy(ts.data(), h->ts, sizeof(TrackState) * h->n_tracks, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "reading track state");
  bool degen = false;
  for (int t = 0; t < h->n_tracks; ++t) {
    if (xhat)
      for (int d = 0; d < 5; ++d) xhat[t * 5 + d] = ts[t].xhat[d];
    if (logZ) logZ[t] = ts[t].log_Z;
    degen |= (ts[t].flags & 1) != 0;
  }
  if (degen) return fail(h, PF_ERR_DEGENERATE, "a track lost all particle weight");
  return PF_OK;
}

// p is null, or page-locked host memory the device can address (cudaHostAlloc
// or cudaHostRegister on a unified address space): *dev = its device address.
// Pageable memory (or a failed query, whose error is cleared) gives false.
static bool host_mapped(void* p, void** dev) {
  *dev = nullptr;
  if (!p) return true;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
  *dev = at.devicePointer;
  return true;
}

pf_status pf_estimate_async(pf_handle* h, float* xhat, double* logZ, void* stream) {
  NvtxRange nvtx_range("pf_estimate_async");
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (!xhat && !logZ) return fail(h, PF_ERR_ARG, "no output buffer");
  if (h->steps_run == 0) return fail(h, PF_ERR_STATE, "no step has run");
  if (h->failed) return fail(h, PF_ERR_STATE, "handle failed earlier: " + h->err);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  // page-locked host buffers: the finishing kernel stores the values itself
  float* xhat_dev = nullptr;
  double* logZ_dev = nullptr;
  if (host_mapped(xhat, reinterpret_cast<void**>(&xhat_dev)) &&
      host_mapped(logZ, reinterpret_cast<void**>(&logZ_dev))) {
    if ((e = launch_finish_out(global_args(h, 1), h->n_tracks, xhat_dev, logZ_dev, h->pdl, s)) != cudaSuccess)
      return cuda_fail(h, e, "k_finish_out");
    h->finish_pending = false;
    h->last_stream = s;
    return PF_OK;
  }
  if (h->finish_pending) {
    if ((e = launch_finish(global_args(h, 1), h->n_tracks, s)) != cudaSuccess) return cuda_fail(h, e, "k_finish");
    h->finish_pending = false;
  }
  // one strided copy per field across the tracks' states
  if (xhat && (e = cudaMemcpy2DAsync(xhat, 5 * sizeof(float), &h->ts[0].xhat[0], sizeof(TrackState), 5 * sizeof(float),
                                     h->n_tracks, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(h, e, "copying estimates");
  if (logZ && (e = cudaMemcpy2DAsync(logZ, sizeof(double), &h->ts[0].log_Z, sizeof(TrackState), sizeof(double),
                                     h->n_tracks, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(h, e, "copying log Z");
  h->last_stream = s;
  return PF_OK;
}

static pf_status check_step(pf_handle* h, int track, int step) {
  if (track < 0 || track >= h->n_tracks) return fail(h, PF_ERR_ARG, "track out of range");
  if (step < 0 || step >= h->steps_run) return fail(h, PF_ERR_STATE, "step has not run");
  if (step < h->steps_run - h->history) return fail(h, PF_ERR_STATE, "step is older than the kept history");
  return PF_OK;
}

pf_status pf_exchange_stats(pf_handle* h, int32_t track, int32_t step, pf_step_stats* out, int32_t* ring_host,
                            double* logW_host, float* xhat_host, float* ess_host) {
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  pf_status st = check_step(h, track, step);
  if (st != PF_OK) return st;
  if ((st = sync(h)) != PF_OK) return st;
  const TrackParams& P = h->tp[track];
  const int slot = step % h->history;
  HistRec r{};
  cudaError_t e = cudaMemcpy(&r, h->hist + P.hist_off + slot, sizeof r, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "reading history");
  if (r.step != step) return fail(h, PF_ERR_STATE, "history slot holds another step");
  if (out) {
    out->step = r.step;
    out->n_ex = r.n_ex;
    out->pe_eff = r.pe_eff;
    out->log_c = r.log_c;
    out->log_Z = r.log_Z;
    for (int d = 0; d < 5; ++d) out->xhat[d] = r.xhat[d];
    out->degenerate_groups = r.degenerate;
    out->resampled_groups = r.resampled;
  }
  if (ring_host || logW_host || xhat_host || ess_host) {
    std::vector<GroupHist> gh(P.G);
    e = cudaMemcpy(gh.data(), h->ghist + P.ghist_off + (long long)slot * P.G, sizeof(GroupHist) * P.G,
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "reading group history");
    for (int m = 0; m < P.G; ++m) {
      if (ring_host) ring_host[m] = gh[m].ring;
      if (logW_host) logW_host[m] = (double)gh[m].logW;
      if (xhat_host)
        for (int d = 0; d < 5; ++d) xhat_host[d * P.G + m] = gh[m].xs[d];
      if (ess_host) ess_host[m] = gh[m].ess;
    }
  }
  return PF_OK;
}

pf_status pf_history(pf_handle* h, int32_t track, int32_t first, int32_t count, pf_step_stats* out) {
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (!out || count < 0) return fail(h, PF_ERR_ARG, "bad output");
  for (int i = 0; i < count; ++i) {
    pf_status st = pf_exchange_stats(h, track, first + i, out + i, nullptr, nullptr, nullptr, nullptr);
    if (st != PF_OK) return st;
  }
  return PF_OK;
}

pf_status pf_particles(pf_handle* h, int32_t track, float* states, uint32_t* anc, float* logw, uint32_t* parent,
                       void* stream) {
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (track < 0 || track >= h->n_tracks) return fail(h, PF_ERR_ARG, "track out of range");
  if (h->steps_run == 0) return fail(h, PF_ERR_STATE, "no step has run");
  const TrackParams& P = h->tp[track];
  if (parent && !P.record) return fail(h, PF_ERR_STATE, "parents are kept only with record_ancestors");
  const int k = h->steps_run - 1;
  const long long Nt = (long long)P.G * P.Np;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (states && (e = launch_export_states(h->pv[k & 1] + P.part_off, h->In[k & 1] + P.part_off, Nt, states, s)))
    return cuda_fail(h, e, "export states");
  const uint32_t* anc_k = h->anc + (long long)(k & 1) * h->N_total;  // step k resampled into buffer k & 1
  if (anc && (e = cudaMemcpyAsync(anc, anc_k + P.part_off, sizeof(uint32_t) * Nt, cudaMemcpyDeviceToDevice, s)))
    return cuda_fail(h, e, "copy ancestors");
  if (logw && (e = cudaMemcpyAsync(logw, h->lw + (h->carry_any ? (k & 1) * lw_stride(h->N_total) : 0) + P.part_off, sizeof(float) * Nt,
                                   cudaMemcpyDeviceToDevice, s)))
    return cuda_fail(h, e, "copy log-weights");
  if (parent &&
      (e = cudaMemcpyAsync(parent, h->parent + P.parent_off + (long long)(k % h->history) * Nt, sizeof(uint32_t) * Nt,
                           cudaMemcpyDeviceToDevice, s)))
    return cuda_fail(h, e, "copy parents");
  return PF_OK;
}

// Standalone resampler: workspace = DevState | GroupDesc[G] | GroupState[G].
static size_t resample_ws(int G) {
  return align_up(sizeof(DevState)) + align_up(sizeof(GroupDesc) * G) + align_up(sizeof(GroupState) * G);
}

pf_status pf_resample_workspace(int32_t G, int32_t Np, size_t* bytes) {
  if (!bytes) return fail(nullptr, PF_ERR_ARG, "bytes is NULL");
  if (G < 1 || Np < 1 || Np > (1 << 20) || (long long)G * Np >= (1ll << 31))
    return fail(nullptr, PF_ERR_ARG, "bad G or Np");
  *bytes = resample_ws(G);
  return PF_OK;
}

pf_status pf_resample(const float* logw, const uint32_t* u, int32_t G, int32_t Np, uint32_t* anc, uint64_t* q,
                      void* workspace, size_t bytes, void* stream) {
  if (!logw || !u || !anc || !workspace) return fail(nullptr, PF_ERR_ARG, "NULL pointer");
  if (G < 1 || Np < 1 || Np > (1 << 20) || (long long)G * Np >= (1ll << 31))
    return fail(nullptr, PF_ERR_ARG, "bad G or Np");
  if ((uintptr_t)workspace % ALIGN) return fail(nullptr, PF_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < resample_ws(G)) return fail(nullptr, PF_ERR_WORKSPACE, "workspace too small");
  char* w = (char*)workspace;
  DevState* ds = (DevState*)w;
  GroupDesc* gd = (GroupDesc*)(w + align_up(sizeof(DevState)));
  GroupState* gs = (GroupState*)(w + align_up(sizeof(DevState)) + align_up(sizeof(GroupDesc) * G));
  std::vector<GroupDesc> h(G);
  for (int g = 0; g < G; ++g) {
    h[g] = GroupDesc{};
    h[g].base = (long long)g * Np;
    h[g].Np = Np;
    h[g].g = g;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ds, 0, sizeof(DevState), s)) ||
      (e = cudaMemcpyAsync(gd, h.data(), sizeof(GroupDesc) * G, cudaMemcpyHostToDevice, s)))
    return cuda_fail(nullptr, e, "pf_resample setup");
  ResampleArgs ra{gd, gs, nullptr, logw, nullptr, anc, 0, (unsigned long long*)q, u, 1, make_qc(), ds};
  ra.n_groups = G;
  ra.max_np = Np;
  ra.lean = q ? 0 : 1;  // without codes to store, the lean instance when the chunks fit
  if ((e = launch_resample(ra, G, resample_cluster(Np, true), false, s)) != cudaSuccess)
    return cuda_fail(nullptr, e, "k_resample");
  return PF_OK;
}

pf_status pf_resample_check(const void* workspace, void* stream) {
  const DevState* src = (const DevState*)workspace;
  if (!src) {
    const int st = noalloc_error_word(&src);
    if (st != PF_OK) return (pf_status)st;
  } else if ((uintptr_t)workspace % ALIGN) {
    return fail(nullptr, PF_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  }
  cudaStream_t s = (cudaStream_t)stream;
  DevState ds{};
  cudaError_t e;
  if ((e = cudaMemcpyAsync(&ds, src, sizeof ds, cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s)))
    return cuda_fail(nullptr, e, "pf_resample_check");
  if (ds.err) {
    char b[200];
    std::snprintf(b, sizeof b, "the resampler reported error bits 0x%x (info %u %u %u)", ds.err, ds.err_info[0],
                  ds.err_info[1], ds.err_info[2]);
    return fail(nullptr, (ds.err & ERR_TIMEOUT) ? PF_ERR_TIMEOUT : PF_ERR_DEVICE, b);
  }
  return PF_OK;
}

pf_status pf_set_theta(pf_handle* h, int32_t track, const float* theta) {
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (track < 0 || track >= h->n_tracks) return fail(h, PF_ERR_ARG, "track out of range");
  if (!theta) return fail(h, PF_ERR_ARG, "theta is NULL");
  const float spsf = theta[PF_THETA_SIGMA_PSF], A = theta[PF_THETA_AMPLITUDE], b = theta[PF_THETA_BACKGROUND];
  const float spos = theta[PF_THETA_SIGMA_POS], sv = theta[PF_THETA_SIGMA_V];
  if (!(std::isfinite(spsf) && spsf > 0.0f) || !std::isfinite(A) || !std::isfinite(b) || !finite_nonneg(spos) ||
      !finite_nonneg(sv))
    return fail(h, PF_ERR_ARG, "theta out of range (sigma_psf > 0, sigma_pos, sigma_v >= 0, all finite)");
  pf_track_config& c = h->cfg[track];
  c.sigma_psf = spsf;
  c.init_state[4] = A;
  c.background = b;
  c.sigma_pos = spos;
  c.sigma_v = sv;
  TrackParams& P = h->tp[track];
  P.spsf = spsf;
  P.c_psf = (float)(1.4426950408889634 / (2.0 * (double)spsf * (double)spsf));
  P.kappa = (float)std::exp2(-2.0 * (double)P.c_psf);
  P.init_state[4] = A;
  P.bg = b;
  P.spos = spos;
  P.sv = sv;
  cudaError_t e = cudaMemcpy(h->trk + track, &P, sizeof(TrackParams), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "uploading track parameters");
  return PF_OK;
}

pf_status pf_reset(pf_handle* h, void* stream) {
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->ds, 0, sizeof(DevState), s)) ||
      (e = cudaMemsetAsync(h->ts, 0, sizeof(TrackState) * h->n_tracks, s)) ||
      (e = cudaMemsetAsync(h->gs, 0, sizeof(GroupState) * h->G_total, s)) ||
      (e = cudaMemsetAsync(h->tile_ctr, 0, sizeof(int), s)) ||
      (e = cudaMemsetAsync(h->fsync, 0, sizeof(unsigned int) * FusedSync{h->G_total}.count(), s)) ||
      (e = cudaMemsetAsync(h->rq, 0, sizeof(unsigned int) * 4 * (size_t)h->n_chunks, s)))
    return cuda_fail(h, e, "pf_reset");
  InitArgs ia{h->trk, h->tiles, h->n_tiles, h->N_total, nullptr, h->pv[1], h->In[1]};
  for (int t = 0; t < h->n_tracks; ++t)
    if (h->cfg[t].init_kind == PF_INIT_USER) return fail(h, PF_ERR_STATE, "pf_reset cannot redraw a user population");
  if ((e = launch_init(ia, h->k1_grid, s)) != cudaSuccess) return cuda_fail(h, e, "k_init");
  if ((e = launch_global(global_args(h, 0), h->n_tracks, s)) != cudaSuccess) return cuda_fail(h, e, "k_global");
  h->steps_run = 0;
  h->finish_pending = false;
  h->failed = 0;
  h->replay_invalid = false;
  h->last_stream = s;
  return PF_OK;
}

pf_status pf_set_replay(pf_handle* h, const uint32_t* parents_dev, int32_t T, void* stream) {
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (!h->adjoint) return fail(h, PF_ERR_STATE, "pf_set_replay needs record_ancestors on every track");
  if (!parents_dev) return fail(h, PF_ERR_ARG, "parents_dev is NULL");
  if (T < 1 || T != h->steps_run) return fail(h, PF_ERR_STATE, "T must equal the number of steps run");
  if (T > h->history) return fail(h, PF_ERR_STATE, "T exceeds the kept history");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  int bad = 0;
  if ((e = cudaMemsetAsync(h->replay_bad, 0, sizeof(int), s)) ||
      (e = launch_set_replay(h->trk, h->tiles, h->n_tiles, parents_dev, h->N_total, h->parent, h->history, T,
                             h->replay_bad, h->k1_grid, s)) ||
      (e = cudaMemcpyAsync(&bad, h->replay_bad, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(h, e, "pf_set_replay");
  h->last_stream = s;
  if (bad) {
    h->replay_invalid = true;
    return fail(h, PF_ERR_ARG, std::to_string(bad) + " parent indices outside their track; pf_backward refuses "
                                                     "this ancestry until a valid pf_set_replay or pf_reset");
  }
  h->replay_invalid = false;
  return PF_OK;
}

pf_status pf_backward(pf_handle* h, const float* const* frames_host, int32_t T, const float* dlogZ_host,
                      float* grad_dev, double* logZ_dev, void* stream) {
  NvtxRange nvtx_range("pf_backward");
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (!h->adjoint) return fail(h, PF_ERR_STATE, "pf_backward needs record_ancestors on every track");
  for (int t = 0; t < h->n_tracks; ++t)
    if (h->tp[t].resample_rule != PF_RESAMPLE_ALWAYS)
      return fail(h, PF_ERR_ARG, "pf_backward needs resample_rule PF_RESAMPLE_ALWAYS on every track");
  if (!frames_host || !dlogZ_host || !grad_dev) return fail(h, PF_ERR_ARG, "NULL argument");
  if (T < 1 || T != h->steps_run) return fail(h, PF_ERR_STATE, "T must equal the number of steps run");
  if (T > h->history) return fail(h, PF_ERR_STATE, "T exceeds the kept history");
  if (h->replay_invalid) return fail(h, PF_ERR_STATE, "the ancestry given to pf_set_replay was rejected");
  for (int i = 0; i < T * h->n_tracks; ++i)
    if (!frames_host[i]) return fail(h, PF_ERR_ARG, "NULL frame pointer");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const long long N = h->N_total;
  const int C = adjoint_segment(T);
  const int nseg = (T + C - 1) / C;
  const int G = h->G_total;
  auto slot_pv = [&](int i) { return h->rp_pv + (long long)i * N; };
  auto slot_I = [&](int i) { return h->rp_I + (long long)i * N; };
  auto ck_pv = [&](int i) { return h->ck_pv + (long long)i * N; };
  auto ck_I = [&](int i) { return h->ck_I + (long long)i * N; };
  if ((e = cudaMemsetAsync(h->grad, 0, sizeof(double) * 5 * h->n_tracks, s)) ||
      (e = cudaMemsetAsync(h->logz_rp, 0, sizeof(double) * h->n_tracks, s)) ||
      (e = cudaMemsetAsync(h->Dacc, 0, sizeof(double) * G, s)) ||
      (e = cudaMemsetAsync(h->ca_pv[0], 0, sizeof(float4) * N, s)) ||
      (e = cudaMemsetAsync(h->ca_pv[1], 0, sizeof(float4) * N, s)) ||
      (e = cudaMemsetAsync(h->ca_I[0], 0, sizeof(float) * N, s)) ||
      (e = cudaMemsetAsync(h->ca_I[1], 0, sizeof(float) * N, s)) ||
      (e = cudaMemcpyAsync(h->seed, dlogZ_host, sizeof(float) * h->n_tracks, cudaMemcpyHostToDevice, s)))
    return cuda_fail(h, e, "pf_backward setup");
  const int grid = h->k1_grid;
  // forward replay with the recorded ancestry; checkpoints every C steps
  InitArgs ia{h->trk, h->tiles, h->n_tiles, N, nullptr, slot_pv(0), slot_I(0)};
  if ((e = launch_init(ia, grid, s)) != cudaSuccess) return cuda_fail(h, e, "k_init");
  for (int k = 0; k < T; ++k) {
    if ((e = prep_frames(h, frames_host + (long long)k * h->n_tracks, s, false)) != cudaSuccess)
      return cuda_fail(h, e, "k_frame_prep");
    ReplayArgs ra{};
    ra.trk = h->trk; ra.tiles = h->tiles; ra.n_tiles = h->n_tiles; ra.parent = h->parent; ra.history = h->history;
    ra.k = k;
    ra.pv_in = k >= 1 ? slot_pv((k - 1) & 1) : nullptr;
    ra.I_in = k >= 1 ? slot_I((k - 1) & 1) : nullptr;
    ra.pv_out = slot_pv(k & 1);
    ra.I_out = slot_I(k & 1);
    ra.ck_pv = (k % C == 0) ? ck_pv(k / C) : nullptr;
    ra.ck_I = (k % C == 0) ? ck_I(k / C) : nullptr;
    ra.weights = 1;
    ra.ypad = h->ypad;
    ra.lbar_prev = k >= 1 ? h->lbar_hist + (long long)(k - 1) * G : nullptr;
    ra.tile_part = h->tile_part;
    if ((e = launch_replay(ra, h->R, grid, s)) != cudaSuccess) return cuda_fail(h, e, "k_replay");
    ReplayGroupArgs rg{h->trk, h->gd, h->tile_part, k, G, h->lam_hist, h->lbar_hist, h->logz_rp, h->dlam, h->seed,
                       k == T - 1 ? 1 : 0};
    if ((e = launch_replay_groups(rg, h->n_tracks, h->max_G, s)) != cudaSuccess)
      return cuda_fail(h, e, "k_replay_groups");
  }
  // reverse sweep, segment by segment, states recomputed from checkpoints
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int k0 = sg * C, k1 = (k0 + C < T) ? k0 + C : T;
    for (int k = k0 + 1; k < k1; ++k) {
      ReplayArgs ra{};
      ra.trk = h->trk; ra.tiles = h->tiles; ra.n_tiles = h->n_tiles; ra.parent = h->parent;
      ra.history = h->history; ra.k = k;
      ra.pv_in = (k - 1 == k0) ? ck_pv(sg) : slot_pv(k - 1 - k0);
      ra.I_in = (k - 1 == k0) ? ck_I(sg) : slot_I(k - 1 - k0);
      ra.pv_out = slot_pv(k - k0);
      ra.I_out = slot_I(k - k0);
      ra.weights = 0;
      ra.ypad = h->ypad;
      ra.tile_part = h->tile_part;
      if ((e = launch_replay(ra, h->R, grid, s)) != cudaSuccess) return cuda_fail(h, e, "k_replay");
    }
    for (int k = k1 - 1; k >= k0; --k) {
      if ((e = prep_frames(h, frames_host + (long long)k * h->n_tracks, s, false)) != cudaSuccess)
        return cuda_fail(h, e, "k_frame_prep");
      AdjointArgs aa{};
      aa.trk = h->trk; aa.tiles = h->tiles; aa.n_tiles = h->n_tiles; aa.parent = h->parent;
      aa.history = h->history; aa.k = k;
      aa.pv = (k == k0) ? ck_pv(sg) : slot_pv(k - k0);
      aa.In = (k == k0) ? ck_I(sg) : slot_I(k - k0);
      aa.ypad = h->ypad;
      aa.lbar_prev = k >= 1 ? h->lbar_hist + (long long)(k - 1) * G : nullptr;
      aa.lam_k = h->lam_hist + (long long)k * G;
      aa.dlam_k = h->dlam;
      aa.D = h->Dacc;
      aa.Cc_pv = h->ca_pv[k & 1];
      aa.Cc_I = h->ca_I[k & 1];
      aa.Cp_pv = h->ca_pv[(k + 1) & 1];
      aa.Cp_I = h->ca_I[(k + 1) & 1];
      aa.grad = h->grad;
      if ((e = launch_adjoint(aa, h->R, grid, s)) != cudaSuccess) return cuda_fail(h, e, "k_adjoint");
      if ((e = launch_adjoint_groups(h->dlam, h->Dacc, G, s)) != cudaSuccess) return cuda_fail(h, e, "k_adjoint_groups");
    }
  }
  if ((e = launch_grad_out(h->grad, h->logz_rp, grad_dev, logZ_dev, h->n_tracks, s)) != cudaSuccess)
    return cuda_fail(h, e, "gradient output");
  h->last_stream = s;
  return PF_OK;
}

pf_status pf_profile_enable(pf_handle* h, int32_t enable) {
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  h->prof = enable ? 1 : 0;
  return PF_OK;
}

pf_status pf_profile_read(pf_handle* h, int32_t n, int64_t* launches, double* total_ms) {
  if (!h) return fail(nullptr, PF_ERR_ARG, "handle is NULL");
  if (n < 0 || n > PF_KERNEL_COUNT) return fail(h, PF_ERR_ARG, "n out of range");
  for (int i = 0; i < PF_KERNEL_COUNT; ++i) {
    const std::vector<cudaEvent_t>& v = h->ev[i];
    double ms = 0.0;
    for (size_t j = 0; j + 1 < v.size(); j += 2) {
      cudaError_t e = cudaEventSynchronize(v[j + 1]);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
      float t = 0.0f;
      if ((e = cudaEventElapsedTime(&t, v[j], v[j + 1])) != cudaSuccess) return cuda_fail(h, e, "elapsed time");
      ms += t;
    }
    if (i < n) {
      if (launches) launches[i] = (int64_t)(v.size() / 2);
      if (total_ms) total_ms[i] = ms;
    }
  }
  for (auto& v : h->ev) {
    for (cudaEvent_t e : v) cudaEventDestroy(e);
    v.clear();
  }
  return PF_OK;
}

// Checkpoint: a header, then the workspace except the TMA descriptors.
struct CheckpointHeader {
  unsigned long long magic, sig, ws_total;
  int32_t abi, steps_run, finish_pending, k1_grid, rs_cluster, rs_threads;
};
static const unsigned long long kCheckpointMagic = 0x6b70635f666e7270ull;  // "prnf_cpk"

pf_status pf_checkpoint_bytes(const pf_handle* h, size_t* bytes) {
  if (!h || !bytes) return fail(nullptr, PF_ERR_ARG, "NULL argument");
  *bytes = sizeof(CheckpointHeader) + h->ws_total - h->tmap_bytes;
  return PF_OK;
}

pf_status pf_save(pf_handle* h, void* host, size_t bytes, void* stream) {
  if (!h || !host) return fail(h, PF_ERR_ARG, "NULL argument");
  size_t need = 0;
  pf_checkpoint_bytes(h, &need);
  if (bytes < need) return fail(h, PF_ERR_ARG, "checkpoint buffer too small");
  cudaStream_t s = (cudaStream_t)stream;
  CheckpointHeader hd{kCheckpointMagic, h->cfg_sig, h->ws_total, PF_ABI_VERSION, h->steps_run,
                      h->finish_pending ? 1 : 0, h->k1_grid, h->rs_cluster, h->rs_threads};
  std::memcpy(host, &hd, sizeof hd);
  char* dst = (char*)host + sizeof hd;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dst, h->ws, h->tmap_off, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(dst + h->tmap_off, h->ws + h->tmap_off + h->tmap_bytes,
                           h->ws_total - h->tmap_off - h->tmap_bytes, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(h, e, "pf_save");
  return PF_OK;
}

pf_status pf_load(pf_handle* h, const void* host, size_t bytes, void* stream) {
  if (!h || !host) return fail(h, PF_ERR_ARG, "NULL argument");
  size_t need = 0;
  pf_checkpoint_bytes(h, &need);
  CheckpointHeader hd{};
  if (bytes < sizeof hd) return fail(h, PF_ERR_ARG, "not a checkpoint");
  std::memcpy(&hd, host, sizeof hd);
  if (hd.magic != kCheckpointMagic || hd.abi != PF_ABI_VERSION) return fail(h, PF_ERR_ARG, "not a checkpoint");
  if (hd.sig != h->cfg_sig || hd.ws_total != h->ws_total || bytes < need)
    return fail(h, PF_ERR_ARG, "checkpoint of a filter with other configurations");
  cudaStream_t s = (cudaStream_t)stream;
  const char* src = (const char*)host + sizeof hd;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h->ws, src, h->tmap_off, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(h->ws + h->tmap_off + h->tmap_bytes, src + h->tmap_off,
                           h->ws_total - h->tmap_off - h->tmap_bytes, cudaMemcpyHostToDevice, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(h, e, "pf_load");
  h->steps_run = hd.steps_run;
  h->finish_pending = hd.finish_pending != 0;
  h->k1_grid = hd.k1_grid;
  h->rs_cluster = hd.rs_cluster;
  h->rs_threads = hd.rs_threads == RS_THREADS_SMALL ? RS_THREADS_SMALL : RS_THREADS;
  h->failed = 0;
  h->last_stream = s;
  if (h->graph) {  // a captured step may hold other launch shapes
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return PF_OK;
}

void pf_destroy(pf_handle* h) { delete h; }

const char* pf_last_error(const pf_handle* h) { return h ? h->err.c_str() : g_err.c_str(); }

}  // extern "C"
