// pf_device.cuh -- device-side data layout and helpers of libpfarna.
//
// Paper: Demirel et al., "An Adaptive Distributed Resampling Algorithm with
// Non-Proportional Allocation" (arXiv:1310.4624).  The paper's M processing
// elements are G groups of Np particles; one track = one filter.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace pf {

// ---------------------------------------------------------------- constants
constexpr int K1_THREADS = 256;       // threads of the propagate/weight kernel
#ifndef PF_K1_PPT
#define PF_K1_PPT 2
#endif
constexpr int K1_PPT = PF_K1_PPT;     // particles per thread
constexpr int K1_TILE = K1_THREADS * K1_PPT;  // slots per tile (one group)
#ifndef PF_K1_MIN_BLOCKS
#define PF_K1_MIN_BLOCKS 4
#endif
constexpr int K1_MIN_BLOCKS = PF_K1_MIN_BLOCKS;  // resident propagate CTAs per SM the register budget targets
constexpr int ROI_W = 40;             // staged frame box width = smem row pitch (floats, = 8 mod 32 banks)
constexpr int ROI_BOX_H = 8;          // rows per TMA box
constexpr int ROI_MAX_BOXES = 8;      // boxes per staged box
constexpr int ROI_ROWS = ROI_BOX_H * ROI_MAX_BOXES;  // staged rows at most (64)
constexpr int ROI_FLOATS = ROI_W * ROI_ROWS;
constexpr int RING_SMEM_G = ROI_FLOATS / 2;  // ring orders drawn ahead up to this G
constexpr int RS_THREADS = 512;       // resampler CTA
constexpr int RS_THREADS_SMALL = 128; // resampler CTA for groups of at most RS_THREADS_SMALL x RS_ITEMS slots
constexpr int RS_ITEMS = 8;           // items per thread per resampler sub-chunk
constexpr int RS_SUB = RS_THREADS * RS_ITEMS;
constexpr int RS_WIN = 2 * RS_SUB;    // resampler merge window: items and outputs merged at once (ancestors staged)
__host__ __device__ constexpr int pad8(int i) { return i + (i >> 3); }  // shared index with one spare per 8
constexpr int RS_SUB_PAD = pad8(RS_SUB);
constexpr int RS_CHUNK = K1_THREADS * RS_ITEMS;  // fused step: items of one resampling chunk (A and B tasks)
constexpr int TASK_P = 0, TASK_A = 1, TASK_B = 2;  // fused step task kinds
constexpr int GL_THREADS = 1024;      // per-track global-step CTA, one thread per group
constexpr int MAX_G = GL_THREADS;      // groups per track
constexpr int MAX_FRAMES_PER_LAUNCH = 1024;

// Philox stream ids (counter word 3 = track << 8 | stream << 4 | call).
constexpr uint32_t ST_INIT = 0, ST_PROP = 1, ST_RESAMPLE = 2, ST_RING = 3, ST_EXCH = 4;
constexpr int TOPO_RING = 0, TOPO_NODE_RING = 1, TOPO_HYPERCUBE = 2;

// Device error word bits.
constexpr uint32_t ERR_INDEX = 1u, ERR_TIMEOUT = 2u, ERR_INVARIANT = 4u, ERR_DRAW = 8u;
constexpr uint32_t ERR_DEBUG = 16u;  // PF_DEBUG build: an index check failed (info: site, index, bound)

enum : int { MODE_RNA = 0, MODE_ARNA = 1 };
enum : int { INIT_POINT = 0, INIT_UNIFORM = 1, INIT_SHARING = 2, INIT_USER = 3 };

// ------------------------------------------------------------- data layout
// Read-only per-track parameters, built on the host at init.
struct TrackParams {
  int G, Np, H, W;
  int mode, init_kind;
  float spsf, bg, sobs, spos, sv, sI;
  float ex_ratio, cutoff;
  float c_psf;      // log2(e) / (2 sigma_psf^2): gx(u) = 2^(-c_psf (u-x)^2)
  float inv2so2;    // 1 / (2 sigma_obs^2)
  float kappa;      // 2^(-2 c_psf): ratio of successive Gaussian ratios
  unsigned long long m_Np;  // fast-division reciprocal of Np
  uint32_t key0, key1, tag;   // Philox key; tag = track_id << 8
  uint32_t rk[20];            // Philox round keys key0 + r W0, key1 + r W1 (r = 0..9), interleaved
  int record;
  int obs_model;              // 0: patch residual, 1: frame likelihood ratio
  int resample_rule;          // 0: every step, 1: Alg. 1's N_eff test per group
  uint32_t ess_t;             // N_thresh = ess_t Np / 2^16
  int send_rule;              // 0: systematic send slots, 1: keyed permutation (Sec. III-C)
  int topology;               // 0: ring, 1: node-aware ring, 2: hypercube (Sec. VI)
  int node_groups;            // topology 1: groups per node
  int hyper_dims;             // ceil(log2 G)
  int perm_bits;              // ceil(log2 Np): the keyed permutation's domain bits
  long long part_off;         // first particle of the track (global slot)
  int group_off;              // first group of the track (global group)
  int tile_off;               // first propagate tile of the track
  int tiles_per_group;
  int pitch;                  // padded frame row pitch (floats)
  long long ypad_off;         // padded frame offset (floats)
  int hist_off;               // first history record of the track
  long long ghist_off;        // first per-group history entry of the track
  long long parent_off;       // first ancestry record (slots) of the track
  float init_state[5], init_lo[5], init_hi[5], init_radius;
};

// Mutable per-track state.
struct TrackState {
  int k;             // step to run next
  int n_ex;          // particles each group sends at step k
  int degenerate;    // groups with no weight at the last step
  int flags;         // bit 0: every group degenerate at some step
  double pe_eff;     // PE_eff used for step k
  double log_c;      // last step's log c
  double log_Z;      // sum of log c
  float xhat[5];
  int steps_done;
  unsigned int ticket;       // groups resampled so far in the current step
  int fin_k;                 // last step whose estimate / log Z / history are complete
  int deg_k;                 // degenerate groups of step k - 1
  float lse_k;               // log c of step k - 1 (FP32)
  int res_k;                 // groups that resampled at step k - 1
};

// Per-group state (global group index).
struct GroupState {
  float lambda;         // carried log group weight log W^(m)
  float off;            // log w offset of particles originating here at step k
  int pred;             // group (track-local) that sends to this one at step k
  uint32_t exo;         // exchange offset o_g of step k
  uint32_t u;           // resampling uniform word of step k
  float M;              // group max log-weight (step k)
  int carry;            // 1: the group skipped resampling at step k - 1, its
                        // particles carry their own log-weights into step k
  int carry_next;       // the resampler's decision at step k (becomes carry at
                        // the track's global step, once no step-k reader is left)
  unsigned long long Q; // group total weight code (step k)
  float xs[5];          // group estimate x^^m (step k)
  float ess;            // group ESS (step k)
  // group max log-weight of step k, by step parity: the largest tile
  // maximum as an order-preserving key (float_key ^ 2^31, 0 = none yet),
  // raised by the propagate tiles, cleared by the resampler one step ahead
  uint32_t mkey[2];
  // fused step: the resampling thresholds of step k (Thresholds below)
  unsigned long long th_A, th_F1, th_M;
  uint32_t th_B, th_F0, th_Np;
};

// Static description of a group.
struct GroupDesc {
  long long base;   // global slot of its slot 0
  int Np;
  int track;
  int g;            // track-local group index
  int tile_begin;   // first propagate tile
  int tile_count;
  int chunk_begin;  // first resampling chunk (fused step)
  int chunk_count;
};

// One history record per (track, step).
struct HistRec {
  int step, n_ex;
  double pe_eff, log_c, log_Z;
  float xhat[5];
  int degenerate;
  int resampled;
};

// Per-group history entry.
struct GroupHist {
  float logW;       // log W^(m) after the step
  int ring;         // group at ring position p used at the step
  float xs[5];
  float ess;
};

// Alg. 1's resampling test N_eff < N_thresh on a group's weight codes: with
// c_i = q_i >> 20, s1 = sum c and s2 = sum c^2, N_eff = s1^2 / s2 and
// N_thresh = t Np / 2^16, so the test is 2^16 s1^2 < t Np s2, compared in
// exact 128-bit integers (s1 <= 2^40, s2 <= 2^60, t <= 2^16, Np <= 2^20).
__device__ __forceinline__ bool ess_below(unsigned long long s1, unsigned long long s2, uint32_t Np, uint32_t t) {
  const unsigned long long alo = s1 * s1, ahi = __umul64hi(s1, s1);
  const unsigned long long a_hi = (ahi << 16) | (alo >> 48), a_lo = alo << 16;
  const unsigned long long m = (unsigned long long)t * Np;
  const unsigned long long b_lo = m * s2, b_hi = __umul64hi(m, s2);
  return a_hi < b_hi || (a_hi == b_hi && a_lo < b_lo);
}

struct DevState {
  unsigned int err;
  unsigned int err_info[3];
};

// ------------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, each two 32x32 -> 64
// multiplies and a Weyl bump of the key.
__device__ __forceinline__ uint4 philox(uint32_t k0, uint32_t k1, uint4 c) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = c.x, b = c.z;
    const uint32_t hi0 = __umulhi(0xD2511F53u, a), lo0 = 0xD2511F53u * a;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, b), lo1 = 0xCD9E8D57u * b;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Uniform in (0,1): ((w >> 9) + 1/2) 2^-23 = (w >> 9) 2^-23 + 2^-24, exact
// in FP32 (an odd multiple of 2^-24 below 1), so one fused multiply-add.
__device__ __forceinline__ float u01(uint32_t w) {
  return __fmaf_rn((float)(w >> 9), 1.1920928955078125e-7f, 5.9604644775390625e-8f);
}

// Box-Muller pair from two words: rho (cos, sin) of 2 pi u_b.  The angle is
// evaluated as 2 pi u_b - pi (the sign folded into rho) so the fast sine and
// cosine stay within [-pi, pi].
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& e0, float& e1) {
  const float rho = sqrtf(-2.0f * logf(u01(wa)));
  float s, c;
  __sincosf(fmaf(u01(wb), 6.28318530717958647f, -3.14159265358979323f), &s, &c);
  e0 = -rho * c;
  e1 = -rho * s;
}

// Lemire bounded integer in [0, s) (multiply-shift with rejection, ACM
// TOMACS 2019); returns false when the word must be redrawn.
__device__ __forceinline__ bool bounded(uint32_t w, uint32_t s, uint32_t& out) {
  const unsigned long long m = (unsigned long long)w * s;
  const uint32_t l = (uint32_t)m;
  if (l < s) {
    const uint32_t t = (0u - s) % s;
    if (l < t) return false;
  }
  out = (uint32_t)(m >> 32);
  return true;
}

// Attempt a of stream `stream`, index c0, step k, word 0.  Returns false if
// 64 attempts were rejected (probability < 2^-64 per call for s < 2^31).
__device__ __forceinline__ bool draw_bounded(uint32_t k0, uint32_t k1, uint32_t tag, uint32_t stream,
                                             uint32_t c0, uint32_t k, uint32_t s, uint32_t& out) {
  for (uint32_t a = 0; a < 64; ++a) {
    const uint4 w = philox(k0, k1, make_uint4(c0, a, k, tag | (stream << 4)));
    if (bounded(w.x, s, out)) return true;
  }
  out = 0;
  return false;
}

// ------------------------------------------------------- fast division
// floor(n / d) for n < 2^32 and 1 <= d < 2^32 as the high word of n * M,
// M = ceil(2^64 / d) (Lemire, Kaser, Kurz, "Faster remainder by direct
// computation", 2019: exact when 64 >= 32 + log2 d); d = 1 is passed as
// M = 0 and returns n.
__host__ __device__ inline unsigned long long fastdiv_magic(uint32_t d) {
  return d <= 1 ? 0ull : (~0ull) / d + 1ull;
}
__device__ __forceinline__ uint32_t fastdiv(uint32_t n, unsigned long long M) {
  return M == 0ull ? n : (uint32_t)__umul64hi((unsigned long long)n, M);
}

// ------------------------------------------------------- fixed-point weights
// q = trunc(p 2^(n+40)), z = fl(fl(lw - M) * L2E), n = rint(z), f = z - n,
// p = sum_{d<=7} c_d f^d by FP32 Horner; 0 when z < -40 or NaN.  All
// operations are single IEEE roundings (no contraction), so the code is
// reproducible on any IEEE machine.
struct QuantCoeffs {
  float c[8];
  float l2e;
};

__device__ __forceinline__ unsigned long long quantize(float lw, float M, const QuantCoeffs& qc) {
  const float t = __fsub_rn(lw, M);
  const float z = __fmul_rn(t, qc.l2e);
  if (!(z >= -40.0f)) return 0ull;
  const float n = rintf(z);
  const float f = __fsub_rn(z, n);
  float p = qc.c[7];
#pragma unroll
  for (int d = 6; d >= 0; --d) p = __fmaf_rn(p, f, qc.c[d]);
  // trunc(p 2^(n+40)) with integer shifts of p's significand (p > 0 normal):
  // p = mant 2^(ex - 23), so the code is mant shifted by ex - 23 + n + 40.
  const uint32_t bits = __float_as_uint(p);
  const unsigned long long mant = (bits & 0x7fffffu) | 0x800000u;
  const int sh = (int)((bits >> 23) & 0xffu) - 127 - 23 + (int)n + 40;
  return sh >= 0 ? (mant << sh) : (mant >> (-sh));
}

// FP32 approximation of a 64-bit unsigned value from its two 32-bit halves
// (32-bit conversions only; relative error < 2^-23).
__device__ __forceinline__ float u64_to_float_approx(unsigned long long v) {
  return __fmaf_rn((float)(uint32_t)(v >> 32), 4294967296.0f, (float)(uint32_t)v);
}

// ------------------------------------------------- resampling thresholds
// Output j of a group with total weight code Q, Np outputs and uniform word
// u sits at theta_j = (j 2^32 + u) Q / (Np 2^32) on the prefix-sum axis.
// Prefix sums S are integers, so theta_j < S exactly when T_j < S with
// T_j = floor(theta_j) = j A + F1 + floor((j B + F0) / Np), where
// A = Q div Np, B = Q mod Np, F = floor(u Q / 2^32), F1 = F div Np,
// F0 = F mod Np.  With Np <= 2^20, j B + F0 < 2^41, and the division is the
// high word of a product with ceil(2^64 / Np) (exact: 64 >= 41 + 20).
struct Thresholds {
  unsigned long long A, F1, M;
  uint32_t B, F0, Np;
  float Af, F1f;  // FP32 approximations of Q / Np and F / Np (comparison filter, le)

  __device__ __forceinline__ void init_filter() {
    Af = __fadd_rn((float)A, (float)B / (float)Np);
    F1f = __fadd_rn((float)F1, (float)F0 / (float)Np);
  }

  __device__ __forceinline__ void init(unsigned long long Q, uint32_t np, uint32_t u) {
    Np = np;
    A = Q / np;
    B = (uint32_t)(Q - A * np);
    const unsigned long long F = (unsigned long long)u * (Q >> 32) + (((unsigned long long)u * (uint32_t)Q) >> 32);
    F1 = F / np;
    F0 = (uint32_t)(F - F1 * np);
    M = np > 1 ? (~0ull) / np + 1ull : 0ull;
    init_filter();
  }
  // The same with the divisions by np done through m = ceil(2^64 / np)
  // (fastdiv_magic): q = floor(n m / 2^64) is floor(n / np) or one more
  // (n < 2^64), fixed by one product.
  __device__ __forceinline__ static unsigned long long udiv(unsigned long long n, uint32_t np,
                                                            unsigned long long m) {
    if (np <= 1) return n;
    unsigned long long q = __umul64hi(n, m);
    if (q * np > n) --q;
    return q;
  }
  __device__ __forceinline__ void init_magic(unsigned long long Q, uint32_t np, uint32_t u, unsigned long long m) {
    Np = np;
    M = np > 1 ? m : 0ull;
    A = udiv(Q, np, M);
    B = (uint32_t)(Q - A * np);
    const unsigned long long F = (unsigned long long)u * (Q >> 32) + (((unsigned long long)u * (uint32_t)Q) >> 32);
    F1 = udiv(F, np, M);
    F0 = (uint32_t)(F - F1 * np);
    init_filter();
  }
  __device__ __forceinline__ unsigned long long T(uint32_t j) const {
    const unsigned long long n = (unsigned long long)j * B + F0;
    return (unsigned long long)j * A + F1 + (Np > 1 ? __umul64hi(n, M) : n);
  }
  // S <= T_j, decided in FP32 when the two are far apart and exactly
  // otherwise: T_j = j Q/Np + F/Np - frac in [0, 1) is approximated by
  // fma(j, Af, F1f) within a relative 2^-21 (j < 2^24, a few FP32
  // roundings) and S by its FP32 value within 2^-23, so a gap beyond
  // 1e-6 of the larger plus 2 decides the comparison; the result is always
  // that of the exact form.
  __device__ __forceinline__ bool le(unsigned long long S, uint32_t j) const {
    return le(S, __fmaf_rn((float)(uint32_t)(S >> 32), 4294967296.0f, (float)(uint32_t)S), (float)j);
  }
  // The same with S's FP32 value Sf (as above) and j's, jf (exact: j < 2^24),
  // given by the caller.
  __device__ __forceinline__ bool le(unsigned long long S, float Sf, float jf) const {
    const float Tf = fmaf(jf, Af, F1f);
    const float m = fmaf(fmaxf(Sf, Tf), 1.0e-6f, 2.0f);
    if (Sf + m < Tf) return true;
    if (Sf > Tf + m) return false;
    return S <= T((uint32_t)jf);
  }
};

__device__ __forceinline__ void set_error(DevState* ds, uint32_t bit, uint32_t a, uint32_t b, uint32_t c) {
  if (atomicOr(&ds->err, bit) == 0) {
    ds->err_info[0] = a;
    ds->err_info[1] = b;
    ds->err_info[2] = c;
  }
}

// Index checks of the PF_DEBUG build (the stand-in for a memory checker):
// an index outside [0, n) sets ERR_DEBUG with the site number, the index and
// the bound, and is replaced by 0 so that the access stays in bounds.  Never
// a trap or an assert.  In the normal build the index passes unchanged.
#ifdef PF_DEBUG
__device__ __forceinline__ long long dbg_index(DevState* ds, long long i, long long n, uint32_t site) {
  if (i < 0 || i >= n) {
    set_error(ds, ERR_DEBUG, site, (uint32_t)i, (uint32_t)n);
    return 0;
  }
  return i;
}
#define PF_DBG_INDEX(ds, i, n, site) (::pf::dbg_index((ds), (long long)(i), (long long)(n), (site)))
#else
#define PF_DBG_INDEX(ds, i, n, site) (i)
#endif

}  // namespace pf
