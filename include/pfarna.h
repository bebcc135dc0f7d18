/*
 * pfarna.h -- C ABI of libpfarna, a GB300 (sm_103a) particle filter with
 * distributed resampling by non-proportional allocation, RNA and adaptive
 * RNA (ARNA), after Demirel, Smal, Niessen, Meijering, Sbalzarini, "An
 * Adaptive Distributed Resampling Algorithm with Non-Proportional
 * Allocation" (arXiv:1310.4624).
 *
 * One call of pf_step advances every track of a handle by one time step of
 * the paper's Alg. 3 (ARNA) or Alg. 2 (RNA): ring order (Sec. IV-B), exchange
 * count (Eq. 3, Eq. 4), ring exchange with fixed group sizes (Sec. III-A),
 * renormalisation, propagation and likelihood weighting (Alg. 1 steps P and
 * U), group estimate and weight, per-group systematic resampling, and the
 * global reduction the paper assigns to a master PE.  The paper's M
 * processing elements are G groups of N_p particles inside one GPU.
 *
 * Conventions for every function below:
 *   - Pointers named *_dev are device pointers, *_host are host pointers.
 *   - Particle slot i = g * Np + j (group g, slot j) inside a track; arrays
 *     that span several tracks concatenate the tracks in handle order.
 *   - State vectors are (x, y, vx, vy, I): position in pixels (x = column,
 *     y = row, pixel centres at integer coordinates), velocity in pixels per
 *     frame, spot amplitude.  Device state arrays passed across this ABI are
 *     structure-of-arrays float32, component-major: 5 rows of N floats.
 *   - Frames are H x W float32, row-major, device-resident.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Calls enqueue work and return without synchronising,
 *     except pf_estimate, pf_exchange_stats and pf_history, which copy to the
 *     host and wait for the handle's last stream (pf_estimate_async only
 *     enqueues its copies).
 *   - Every call returns a pf_status; nothing is thrown across the ABI.  On
 *     failure the text of the error is available from pf_last_error.
 *   - The caller owns all device memory (workspace, frames, outputs); the
 *     handle owns only host-side metadata and is freed by pf_destroy.
 *   - Device faults detected by the kernels (bad index, bounded wait
 *     exhausted, internal invariant) set a device error word; it is read and
 *     reported (PF_ERR_DEVICE / PF_ERR_TIMEOUT) by the next call that
 *     synchronises.  A library built with PF_DEBUG also checks the indices
 *     it takes from data (ring entries, exchange sources, mark positions,
 *     patch reads) and reports a failed check the same way, with the site,
 *     the index and the bound in the message.
 */
#ifndef PFARNA_H
#define PFARNA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF_ABI_VERSION 5

typedef enum pf_status {
  PF_OK = 0,
  PF_ERR_ARG = 1,        /* invalid argument (sizes, NULL, unsupported config) */
  PF_ERR_STATE = 2,      /* call out of order (e.g. stats for a step not run) */
  PF_ERR_CUDA = 3,       /* a CUDA runtime call failed */
  PF_ERR_WORKSPACE = 4,  /* workspace too small or misaligned */
  PF_ERR_DEGENERATE = 5, /* every group of a track lost all weight */
  PF_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up */
  PF_ERR_DEVICE = 7      /* a kernel reported an internal error */
} pf_status;

/* Exchange schedule (Sec. III-B, Sec. IV). */
enum { PF_RNA = 0, PF_ARNA = 1 };

/* Initial population (Sec. V, "tracking" and "information sharing"). */
enum {
  PF_INIT_POINT = 0,   /* every particle at init_state */
  PF_INIT_UNIFORM = 1, /* component d uniform in [init_lo[d], init_hi[d]] */
  PF_INIT_SHARING = 2, /* group 0: position uniform in the disc of radius
                          init_radius around init_state, other components of
                          init_state; groups >= 1: as PF_INIT_UNIFORM */
  PF_INIT_USER = 3     /* copied from pf_init's user_state_dev */
};

/* Observation models (obs_model).  Both describe a Gaussian spot of width
 * sigma_psf and amplitude I on background `background` (Sec. V, Fig. 1)
 * with Gaussian noise sigma_obs, the spot truncated to the (2 patch_radius
 * + 1)^2 pixels around the particle's nearest pixel, pixels outside the
 * frame counting as background:
 *  PF_OBS_PATCH: l = -sum_patch (z - b - I gx gy)^2 / (2 sigma_obs^2), the
 *    residual of the patch alone;
 *  PF_OBS_FRAME: the likelihood of the whole frame divided by that of the
 *    background alone, l = -sum_patch [(z - b - I gx gy)^2 - (z - b)^2] /
 *    (2 sigma_obs^2) (pixels off the patch cancel): particles over plain
 *    background score about 0, so a search from a spread-out start finds
 *    the spot (the information-sharing scenario of Sec. V-B); log Z is then
 *    the log of that ratio. */
enum { PF_OBS_PATCH = 0, PF_OBS_FRAME = 1 };

/* When a group resamples (resample_rule).
 *  PF_RESAMPLE_ALWAYS: every group at every step (Alg. 2 / Alg. 3).
 *  PF_RESAMPLE_ESS: Alg. 1's test, per group: group m resamples at step k
 *    only when its effective sample size N_eff = (sum w)^2 / sum w^2 is
 *    below N_thresh = ess_fraction * Np; a group that does not resample
 *    keeps its particles in place with their own weights, which they carry
 *    into the next step (and through the ring exchange).  The test is taken
 *    exactly on the resampler's integer weight codes q: with c_i = q_i >> 20,
 *    resample iff 2^16 (sum c)^2 < t Np sum c^2, t = round(ess_fraction
 *    2^16).  A group without finite weight resamples as the identity. */
enum { PF_RESAMPLE_ALWAYS = 0, PF_RESAMPLE_ESS = 1 };

/* Which slots a group sends (send_rule; Sec. III-C: each PE randomly selects
 * N_ex particles).  A receiver puts the particles into its own send slots,
 * the t-th sent slot of the sender into the t-th send slot of the receiver.
 *  PF_SEND_SYSTEMATIC: slots floor((t Np + o_g) / N_ex), t < N_ex, with a
 *    uniform offset o_g per group and step: every slot with probability
 *    N_ex / Np, spread evenly over the slots.
 *  PF_SEND_KEYED: slots pi_g(t), t < N_ex, of a keyed pseudo-random
 *    permutation of [0, Np) per group and step (a four-round Feistel network
 *    on ceil(log2 Np) bits with cycle walking, round keys from the Philox
 *    stream of the exchange): a uniformly random-looking subset. */
enum { PF_SEND_SYSTEMATIC = 0, PF_SEND_KEYED = 1 };

/* Who exchanges with whom (topology; Sec. IV-B, and Sec. VI's future work).
 *  PF_TOPO_RING: the ring of Alg. 2 (fixed, PF_RNA) or a fresh random ring
 *    every step (PF_ARNA).
 *  PF_TOPO_NODE_RING: groups form nodes of node_groups consecutive groups
 *    (for instance the groups sharing a die or a machine); PF_ARNA's random
 *    ring visits the nodes in a random order and each node's groups in a
 *    random order, so one ring edge per node leaves it.  PF_RNA: the fixed
 *    ring, which already runs node by node.
 *  PF_TOPO_HYPERCUBE: at step k every group exchanges N_ex particles with
 *    its partner g xor 2^d along one dimension d of the ceil(log2 G)-cube (no
 *    exchange for a group whose partner would be >= G); PF_RNA cycles d,
 *    PF_ARNA draws it at random every step.  The ring order reported by
 *    pf_exchange_stats is then each group's partner. */
enum { PF_TOPO_RING = 0, PF_TOPO_NODE_RING = 1, PF_TOPO_HYPERCUBE = 2 };

/* One track's filter.  Observation model: obs_model above.  Dynamics: nearly
 * constant velocity with unit frame interval and independent Gaussian noise
 * sigma_pos (position), sigma_v (velocity), sigma_I (intensity). */
typedef struct pf_track_config {
  int32_t G;            /* groups (the paper's M PEs), 1 .. 1024 */
  int32_t Np;           /* particles per group (N_p = N / M), 1 .. 2^20; G*Np < 2^31 */
  int32_t H, W;         /* frame size, 1 .. 16384 each */
  int32_t patch_radius; /* 1 .. 7; the paper's workloads use 5 (11 x 11) */
  int32_t mode;         /* PF_RNA or PF_ARNA */
  float sigma_psf, background, sigma_obs;
  float sigma_pos, sigma_v, sigma_I;
  float ex_ratio;       /* PF_RNA: N_ex = floor(ex_ratio * Np), ex_ratio in [0, 1] */
  float pe_eff_cutoff;  /* PF_ARNA: no exchange once PE_eff >= cutoff * G (0.99) */
  int32_t init_kind;    /* PF_INIT_* */
  float init_state[5];
  float init_lo[5];
  float init_hi[5];
  float init_radius;
  int32_t obs_model;    /* PF_OBS_PATCH (default) or PF_OBS_FRAME */
  uint64_t seed;        /* Philox4x32-10 key */
  uint32_t track_id;    /* Philox stream id of this track, < 2^24 */
  int32_t record_ancestors; /* 1: keep per-step ancestry for pf_backward */
  int32_t resample_rule;    /* PF_RESAMPLE_ALWAYS (0) or PF_RESAMPLE_ESS */
  float ess_fraction;       /* PF_RESAMPLE_ESS: N_thresh / Np, in [0, 1] */
  int32_t send_rule;        /* PF_SEND_SYSTEMATIC (0) or PF_SEND_KEYED */
  int32_t topology;         /* PF_TOPO_RING (0), PF_TOPO_NODE_RING or PF_TOPO_HYPERCUBE */
  int32_t node_groups;      /* PF_TOPO_NODE_RING: groups per node, >= 1 */
} pf_track_config;

/* Statistics of one completed step of one track. */
typedef struct pf_step_stats {
  int32_t step;              /* k, 0-based */
  int32_t n_ex;              /* particles each group sent at step k */
  double pe_eff;             /* Eq. 4 PE_eff of the weights carried into step k, in [1, G] */
  double log_c;              /* log of the step's incremental likelihood estimate */
  double log_Z;              /* sum of log_c over steps 0 .. k */
  float xhat[5];             /* global estimate x^_k (Alg. 3 step 10) */
  int32_t degenerate_groups; /* groups whose weights were all zero / NaN */
  int32_t resampled_groups;  /* groups that resampled at step k (all of them under PF_RESAMPLE_ALWAYS) */
} pf_step_stats;

typedef struct pf_handle pf_handle;

/* ABI version of the loaded library (PF_ABI_VERSION it was built with). */
int32_t pf_abi_version(void);

/* Workspace bytes needed by pf_init for `n_tracks` configs (cfg[0..n-1]).
 * The paper's problem (Sec. II) is the filtering density of the state given
 * the frames so far, carried by N = G * Np weighted particles split over
 * the G PEs (Sec. III); the workspace holds those particles, their weights
 * and the per-group and per-step quantities of Alg. 3, sized here
 * for `history` steps of statistics (>= 1; the last `history` steps stay
 * readable through pf_exchange_stats / pf_history).  With record_ancestors
 * set, `history` is also the longest sequence pf_backward can differentiate.
 * Errors: PF_ERR_ARG for invalid configs or NULL pointers. */
pf_status pf_query_workspace(const pf_track_config* cfg, int32_t n_tracks, int32_t history,
                             size_t* bytes);

/* Create a filter over `n_tracks` tracks in the caller's device workspace
 * (`bytes` >= pf_query_workspace's answer, 256-byte aligned) and enqueue the
 * draw of the initial population on `stream`.  user_state_dev: for tracks
 * with init_kind == PF_INIT_USER, the initial states as 5 x N_total float32
 * SoA (N_total = sum of G * Np over all tracks; other tracks' columns are
 * ignored), else may be NULL; it is read before pf_init's work completes on
 * the stream.  All tracks of one handle must share patch_radius.  The
 * workspace must stay allocated and untouched until pf_destroy.
 * The step kernels are launched with programmatic dependent launch (each
 * may start while the previous kernel in the stream drains, and waits for
 * its completion before touching memory); the environment variable
 * PFARNA_PDL=0 at pf_init selects plain stream serialisation instead.
 * PFARNA_RS_THREADS=128 or 512 at pf_init forces the resampler's CTA size
 * (by default 128 when every group has at most 1024 particles, else 512).
 * Results are identical either way.  PFARNA_FUSED=1 at pf_init runs each step
 * as one persistent launch instead (propagate + weight tiles, the per-group
 * resampling split into chunk tasks that start as soon as their group's
 * tiles are done, and the global step), with the same results; on the
 * workloads measured it is slower than the two launches, so it is off by
 * default.  PFARNA_TEST_WITHHOLD_COPY=1 at pf_init
 * (failure-detection tests only) makes the propagate kernel issue no
 * frame-staging copy, so its bounded wait (0.2 s) runs out: the step ends
 * early and the next synchronising call reports PF_ERR_TIMEOUT.
 * Errors: PF_ERR_ARG, PF_ERR_WORKSPACE, PF_ERR_CUDA. */
pf_status pf_init(const pf_track_config* cfg, int32_t n_tracks, int32_t history, void* workspace_dev,
                  size_t bytes, const float* user_state_dev, void* stream, pf_handle** out);

/* Enqueue one time step k (Alg. 3, or Alg. 2 for PF_RNA) for every track.
 * frames_host: host array of n_tracks device pointers, frame k of each
 * track (H x W float32); the frames must stay valid until the step has run
 * on `stream`.  At k = 0 there is no propagation and no exchange: the
 * initial population is weighted by frame 0.  A step is two kernels,
 * propagate + weight and resampling, whose last group per track also runs
 * the track's global step (Alg. 3 steps 8-10, and steps 1-2 of the next
 * step); a batch of tracks, or a single track whose frame a TMA descriptor
 * cannot describe, adds a frame-preparation kernel before them.
 * Errors: PF_ERR_ARG (NULL frame), PF_ERR_STATE (handle failed before),
 * PF_ERR_CUDA. */
pf_status pf_step(pf_handle* h, const float* const* frames_host, void* stream);

/* Bytes of the device staging buffer pf_step_host needs: two slots (by step
 * parity), each with every track's H x W float32 frame at a 256-byte
 * aligned offset.  Errors: PF_ERR_ARG. */
pf_status pf_host_staging_bytes(const pf_handle* h, size_t* bytes);

/* pf_step with the frames in HOST memory: frames_host holds n_tracks host
 * pointers (frame k of each track, H x W float32, row-major).  The frames
 * are uploaded on a stream of the handle's own into the caller's device
 * staging buffer (staging_dev: 256-byte aligned, at least
 * pf_host_staging_bytes; the caller owns it and keeps it for the handle's
 * life), slot k & 1, after the step two back has finished reading that
 * slot; `stream` waits for the upload, then runs pf_step on the staged
 * frames.  A host pointer given to several tracks of the same frame size is
 * uploaded once.  With page-locked host frames (cudaHostAlloc,
 * cudaHostRegister) the call returns at once and frame k + 1 uploads while
 * step k runs; the host frame must then stay unchanged until the upload has
 * run (the step's completion on `stream` implies it).  Pageable frames are
 * copied before the call returns.  Errors: PF_ERR_ARG (NULL frame, staging
 * buffer NULL, misaligned or too small), PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_step_host(pf_handle* h, const float* const* frames_host, void* staging_dev, size_t staging_bytes,
                       void* stream);

/* pf_step with the frames taken from a device table: table_dev holds
 * T_table x n_tracks device pointers, frame k of track t at index
 * k * n_tracks + t, and the step's index k is read on the device, so the
 * launch sequence has no per-step parameters.  n_tracks <= 65535.
 * Errors: PF_ERR_ARG, PF_ERR_STATE (no table entry for this step),
 * PF_ERR_CUDA. */
pf_status pf_step_table(pf_handle* h, const float* const* table_dev, int32_t T_table, void* stream);

/* pf_step_table through a CUDA graph: the first call (and the first after
 * the table, T_table or the autotuned shapes change) captures the step's
 * launches into a graph; every call launches it on `stream`.
 * Errors: as pf_step_table. */
pf_status pf_graph_step(pf_handle* h, const float* const* table_dev, int32_t T_table, void* stream);

/* One pf_step that also chooses the launch shapes of the handle's later
 * steps: the propagate kernel's grid (SM count x resident CTAs per SM, 1 ..
 * the occupancy limit) and the resampler's thread-block cluster size
 * (1, 2, 4, 8) and CTA size (512 or 128 threads), each the fastest of the candidates timed with CUDA events
 * on this step's data (the propagate candidates first: it is idempotent
 * until a resampler replaces the ancestors it reads).  Results
 * are cached per problem shape for the process.  Synchronises the stream.
 * k1_grid_out / cluster_out (may be NULL) receive the choices.
 * Errors: PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_autotune(pf_handle* h, const float* const* frames_host, int32_t* k1_grid_out, int32_t* cluster_out,
                      void* stream);

/* Wait for the handle's last stream and copy the latest global estimate
 * (n_tracks x 5 floats, may be NULL) and log marginal-likelihood estimate
 * log Z = sum_k log c_k (n_tracks doubles, may be NULL) to the host.  These
 * are the master PE's outputs of Alg. 3 steps 9-10: the estimate combines
 * the group estimates x^^m (step 6) with the normalised group weights, and
 * c_k is the sum of the group weights W^(m) (the normaliser of step 9).
 * Errors: PF_ERR_STATE (no step run), PF_ERR_DEGENERATE (some track lost all
 * weight: its values are NaN / -inf), PF_ERR_DEVICE / PF_ERR_TIMEOUT (the
 * kernels reported an error), PF_ERR_CUDA. */
pf_status pf_estimate(pf_handle* h, float* xhat_host, double* log_Z_host);

/* pf_estimate without waiting: enqueue on `stream` (the stream the steps
 * run on) the completion of the last step's statistics and copies of x^
 * (n_tracks x 5 floats) and log Z (n_tracks doubles) into the caller's host
 * buffers, and return.  The values are there once the stream has passed
 * this point (the caller's event or synchronisation).  Page-locked host
 * buffers (cudaHostAlloc, cudaHostRegister) are written by the finishing
 * kernel itself through their device addresses, so no copy follows it on
 * the stream; pageable buffers are filled by copies.  Either way a stream
 * of frames can be filtered with the next frame's upload and the last
 * estimate's read-back in flight.  Degenerate tracks and device errors are
 * reported by the next synchronising call.  Errors: PF_ERR_ARG,
 * PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_estimate_async(pf_handle* h, float* xhat_host, double* log_Z_host, void* stream);

/* Statistics of step `step` (< steps run, and among the last `history`) of
 * track `track`: the exchange count N_ex of Eq. 3 (the fixed ratio for
 * PF_RNA) and the PE_eff of Eq. 4 it was decided from, the ring of Sec.
 * IV-B, the group weights and estimates of Alg. 3 steps 6 and 8, and the
 * step's incremental likelihood (steps 9-10).  Optional per-group arrays
 * (length G, may be NULL):
 * ring_host[p] = group at ring position p (group ring[p] sends to
 * ring[(p+1) mod G]) used at that step; group_logW_host = log W^(m) after
 * the step; group_xhat_host = group estimates x^^m, 5 x G SoA;
 * group_ess_host = 1 / sum w^2 within each group.  Waits for the stream.
 * Errors: PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_exchange_stats(pf_handle* h, int32_t track, int32_t step, pf_step_stats* out,
                            int32_t* ring_host, double* group_logW_host, float* group_xhat_host,
                            float* group_ess_host);

/* Statistics of `count` consecutive steps first .. first+count-1 of one
 * track (each among the last `history`).  Waits for the stream.
 * Errors: PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_history(pf_handle* h, int32_t track, int32_t first, int32_t count, pf_step_stats* out);

/* Device-to-device copies, enqueued on `stream`, of the latest step's
 * particles of track `track` (each pointer may be NULL):
 *   states_dev: the propagated states X_k before resampling, 5 x N SoA;
 *   anc_dev:    resampling ancestors, anc[g*Np + j] = slot (within the
 *               track, g*Np + a) whose state slot j of group g copies;
 *   logw_dev:   log w~_k = log of the renormalised prior weight plus the
 *               log-likelihood, the input of the resampler;
 *   parent_dev: the slot of X_{k-1} that each slot was propagated from
 *               (the exchange composed with the previous resampling).
 * Errors: PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_particles(pf_handle* h, int32_t track, float* states_dev, uint32_t* anc_dev,
                       float* logw_dev, uint32_t* parent_dev, void* stream);

/* Workspace bytes for pf_resample on G groups of Np particles. */
pf_status pf_resample_workspace(int32_t G, int32_t Np, size_t* bytes);

/* Per-group systematic resampling (Alg. 1 step 6) of G groups of Np
 * particles, on the GPU kernel pf_step uses, exposed for verification.
 * logw_dev: G*Np float32 log-weights, group-major; u_dev: G uint32 uniform
 * words (the offset is u / 2^32); anc_dev: G*Np uint32 outputs, anc[g*Np+j]
 * = ancestor slot within the group (0 .. Np-1); q_dev: optional G*Np uint64
 * outputs, the fixed-point weight codes the resampler used (may be NULL).
 * Weight codes: with M the group maximum, q = trunc(p 2^(n+40)) where
 * z = fl(fl(lw - M) * fl32(log2 e)), n = rint(z), p = the degree-7 Taylor
 * polynomial of 2^(z-n) in FP32 Horner form; q = 0 when z < -40 or NaN.
 * Output j takes the particle i with S_i <= (j + u/2^32) Q / Np < S_{i+1},
 * S the prefix sums of q and Q their total, compared exactly in 128-bit
 * integers; a group with Q = 0 resamples as the identity.
 * G >= 1, 1 <= Np <= 2^20, G*Np < 2^31.  The call only enqueues: a
 * device-side error of the kernel (an internal bound exhausted, reported in
 * the error word at the start of the workspace) is not returned here but by
 * pf_resample_check(workspace_dev, stream).
 * Errors: PF_ERR_ARG, PF_ERR_WORKSPACE, PF_ERR_CUDA. */
pf_status pf_resample(const float* logw_dev, const uint32_t* u_dev, int32_t G, int32_t Np,
                      uint32_t* anc_dev, uint64_t* q_dev, void* workspace_dev, size_t bytes,
                      void* stream);

/* Largest G pf_resample_noalloc accepts (the size of its fixed scratch). */
#define PF_NOALLOC_MAX_GROUPS 1024

/* pf_resample without a workspace: the same kernel and the same results
 * (logw_dev, u_dev, G, Np, anc_dev, q_dev exactly as for pf_resample), for
 * callers that cannot allocate device memory at the point where they
 * resample -- a fixed memory budget reserved up front, a framework whose
 * caching allocator must not be bypassed, or a latency-critical loop where
 * cudaMalloc's implicit device synchronisation is not acceptable.  The paper
 * has no counterpart; it is a deployment variant of pf_resample.
 * Its scratch (about 96 KB) is a fixed device array in the library, which
 * every GPU that loads the library holds until the process exits.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current) and should come before
 * any stream capture.  The cached address belongs to the CUDA context it was
 * looked up in; after cudaDeviceReset the next call looks it up again.  The
 * call allocates nothing and frees nothing.  All calls share the array,
 * which keeps the last call's contents; each call clears what must start at
 * zero, and calls that overlap on the GPU race.  As with pf_resample, a
 * device-side error of the kernel is not returned by this call but by
 * pf_resample_check(NULL, stream), until the next call clears it.
 * G >= 1 and G <= PF_NOALLOC_MAX_GROUPS, 1 <= Np <= 2^20, G*Np < 2^31;
 * larger G is rejected with PF_ERR_ARG.  Errors are reported through
 * pf_last_error(NULL).  Errors: PF_ERR_ARG, PF_ERR_CUDA. */
pf_status pf_resample_noalloc(const float* logw_dev, const uint32_t* u_dev, int32_t G, int32_t Np,
                              uint32_t* anc_dev, uint64_t* q_dev, void* stream);

/* Wait for `stream` and report the device-side error word of the last
 * pf_resample run in `workspace_dev` (its workspace), or, with workspace_dev
 * NULL, of the last pf_resample_noalloc on the current device: PF_OK, or
 * PF_ERR_DEVICE / PF_ERR_TIMEOUT with the error bits in pf_last_error(NULL).
 * The resampler itself is Alg. 1 step 6; this call only reads back what its
 * kernel recorded.  Errors: PF_ERR_WORKSPACE (misaligned), PF_ERR_CUDA,
 * PF_ERR_DEVICE, PF_ERR_TIMEOUT. */
pf_status pf_resample_check(const void* workspace_dev, void* stream);

/* Kernel timing.  With enable = 1, every later pf_step records a pair of
 * CUDA events around each of its kernels, on the stream it launches them
 * on; enable = 0 stops recording.  Recording adds no synchronisation.
 * Errors: PF_ERR_ARG, PF_ERR_CUDA. */
pf_status pf_profile_enable(pf_handle* h, int32_t enable);

/* Kernels of one step, in launch order, as indexed by pf_profile_read. */
enum {
  PF_KERNEL_FRAME_PREP = 0,
  PF_KERNEL_PROPAGATE_WEIGHT = 1,
  PF_KERNEL_RESAMPLE = 2,
  PF_KERNEL_GLOBAL = 3,
  PF_KERNEL_FUSED_STEP = 4, /* the one-launch step: propagate, weight, resample, global step */
  PF_KERNEL_COUNT = 5
};

/* Wait for the recorded work, then write, for each of the first n (<=
 * PF_KERNEL_COUNT) kernels, the number of recorded launches and their
 * summed device duration in milliseconds; the records are then cleared.
 * Either array may be NULL.  Errors: PF_ERR_ARG, PF_ERR_CUDA. */
pf_status pf_profile_read(pf_handle* h, int32_t n, int64_t* launches, double* total_ms);

/* Parameters of the differentiable form: theta = (sigma_psf, A, b,
 * sigma_pos, sigma_v), A being the initial intensity of the particles
 * (init_state[4]; every particle for PF_INIT_POINT, group 0 for
 * PF_INIT_SHARING). */
enum {
  PF_THETA_SIGMA_PSF = 0,
  PF_THETA_AMPLITUDE = 1,
  PF_THETA_BACKGROUND = 2,
  PF_THETA_SIGMA_POS = 3,
  PF_THETA_SIGMA_V = 4,
  PF_THETA_COUNT = 5
};

/* Set theta (PF_THETA_COUNT floats, host) of one track; later pf_step,
 * pf_reset and pf_backward calls use it.  Synchronous upload.
 * Errors: PF_ERR_ARG (out of range), PF_ERR_CUDA. */
pf_status pf_set_theta(pf_handle* h, int32_t track, const float* theta_host);

/* Restart every track from a fresh initial population drawn with the
 * current parameters (step 0 next); not for PF_INIT_USER tracks.
 * Errors: PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_reset(pf_handle* h, void* stream);

/* Gradient of log Z = sum_{k<T} log c_k with respect to theta, with the
 * resampling ancestry of the T steps run since pf_init / pf_reset held fixed
 * (every track must have record_ancestors; T = steps run <= history).  The
 * forward pass is replayed from the initial population (drawn again with
 * the current theta) through the recorded parents and the same Philox
 * streams, keeping states only at checkpoints every ceil(sqrt(T)) steps;
 * the reverse sweep recomputes each segment's states and back-propagates
 * through the group log-weights (Alg. 3 steps 4-10), the likelihood and the
 * NCV dynamics.  frames_host: T x n_tracks device pointers, frame k of track
 * t at index k * n_tracks + t (the frames of the forward run).
 * dlogZ_host: n_tracks upstream derivatives.  grad_dev: n_tracks x 5 floats,
 * dlogZ * d log Z / d theta.  logZ_dev: optional n_tracks doubles, the
 * replayed log Z.  Enqueued on `stream`; the forward filter state is left
 * as it was.  Tracks must use PF_RESAMPLE_ALWAYS (the replay resamples at
 * every step).  Errors: PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_backward(pf_handle* h, const float* const* frames_host, int32_t T, const float* dlogZ_host,
                      float* grad_dev, double* logZ_dev, void* stream);

/* Replace the recorded ancestry of the T steps run (T must equal the steps
 * run since pf_init / pf_reset, and T <= history) by the caller's, so that
 * pf_backward differentiates log Z along an externally supplied ancestry
 * (for instance another implementation's run, for verification): the
 * replay of Alg. 3 with steps 3 and 7 (exchange and resampling) held fixed
 * at the given choices.  parents_dev: device array of T x N_total uint32,
 * row k (k = 1 .. T-1; row 0 is ignored) holding, for every track in handle
 * order, the track-local slot of X_{k-1} that each slot of step k was
 * propagated from (the exchange composed with the previous step's
 * resampling, as pf_particles' parent_dev reports it); the particle's
 * carried weight is that of the slot's group, slot / Np.  The exchange
 * count and ring of each step are implied by these parents.  Every track
 * needs record_ancestors.  Synchronises `stream`.  An index outside its
 * track is rejected: PF_ERR_ARG, and pf_backward refuses until a valid
 * pf_set_replay or pf_reset.  The forward filter's states are untouched.
 * Errors: PF_ERR_ARG, PF_ERR_STATE, PF_ERR_CUDA. */
pf_status pf_set_replay(pf_handle* h, const uint32_t* parents_dev, int32_t T, void* stream);

/* Checkpoint and resume.  A filter's whole state lives in its workspace
 * and a few host counters, and every random draw is a counter-based Philox
 * word, so a restored filter continues exactly as the saved one would.
 * pf_checkpoint_bytes: the size of a checkpoint of `h`.
 * pf_save: waits for the handle's work on `stream` and copies its state to
 * `host` (bytes >= pf_checkpoint_bytes).
 * pf_load: restores a checkpoint into `h`, which must have been created
 * with the same configurations and history as the saved handle (it may be
 * the same handle); enqueued on `stream` and synchronised.  No counterpart
 * in the paper (its runs are not resumed).
 * Errors: PF_ERR_ARG (NULL, too small, not a checkpoint of a filter of this
 * configuration), PF_ERR_CUDA. */
pf_status pf_checkpoint_bytes(const pf_handle* h, size_t* bytes);
pf_status pf_save(pf_handle* h, void* host, size_t bytes, void* stream);
pf_status pf_load(pf_handle* h, const void* host, size_t bytes, void* stream);

/* Release the handle's host metadata (the workspace stays the caller's). */
void pf_destroy(pf_handle* h);

/* Text of the last error of `h`, or of the calling thread's last failed
 * handle-less call when h is NULL.  Never NULL; valid until the next call. */
const char* pf_last_error(const pf_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* PFARNA_H */
