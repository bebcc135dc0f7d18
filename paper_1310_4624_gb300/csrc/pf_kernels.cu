// pf_kernels.cu -- CUDA kernels (sm_103a) of one RNA / ARNA filter step.
//
// Paper: Demirel et al., "An Adaptive Distributed Resampling Algorithm with
// Non-Proportional Allocation" (arXiv:1310.4624).
//
// One step k of Alg. 3 (Alg. 2 for RNA) is two launches on one stream,
// chained by programmatic dependent launch:
//   k_propagate_weight  ring exchange composed with the previous resampling
//                       (Alg. 3 steps 3-4), propagation (Alg. 1 step P),
//                       likelihood (step U) on frame boxes staged by TMA,
//                       per-tile partial sums for the group estimate (Alg. 3
//                       step 6) and the group maxima; its leading blocks
//                       draw the next step's ring and exchange offsets and
//                       finish the previous step's statistics
//   k_resample          per-group exact systematic resampling on fixed-point
//                       weight codes (Alg. 3 step 7), one thread-block
//                       cluster per group (code totals and the marks of the
//                       ancestor search through distributed shared memory);
//                       the track's global step -- the master PE's
//                       reduction (steps 9-10), the weight carry (step 8),
//                       the next ring order (step 1) and exchange count
//                       (step 2, Eq. 3/4) -- once every group has reported
// A batch of tracks given device frames first pads them (k_frame_prep);
// k_global prepares step 0; k_finish / k_finish_out complete the last
// step's statistics when the host reads them.  The step index lives on the
// device, so the same launch sequence serves every step.
#include <cooperative_groups.h>
#include <mutex>
#include <utility>
#include <cuda.h>
#include <cuda_runtime.h>

#include <climits>

#include <cmath>
#include <cstdint>

#include "pf_device.cuh"
#include "pf_launch.h"
#include "pf_math.cuh"

namespace cg = cooperative_groups;

namespace pf {

// ========================================================= initial population
// Initial population (Sec. V tracking / information-sharing modes), drawn
// from Philox stream INIT into the buffer step 0 reads.
__global__ void __launch_bounds__(K1_THREADS) k_init(InitArgs a) {
  for (int e = blockIdx.x * K1_PPT; e < a.n_tiles * K1_PPT; e += gridDim.x * K1_PPT) {
   for (int q = 0; q < K1_PPT; ++q) {
    const int4 td = a.tiles[(e + q) / K1_PPT];
    const int jj = threadIdx.x + ((e + q) % K1_PPT) * K1_THREADS;
    if (jj >= td.w) continue;
    const TrackParams& P = a.trk[td.x];
    const int g = td.y, j = td.z + jj;
    const long long i = P.part_off + (long long)g * P.Np + j;
    float s[5];
    if (P.init_kind == INIT_USER) {
#pragma unroll
      for (int d = 0; d < 5; ++d) s[d] = a.user[(long long)d * a.n_total + i];
    } else {
      const uint4 w0 = philox(P.key0, P.key1, make_uint4(j, g, 0u, P.tag | (ST_INIT << 4) | 0u));
      const uint4 w1 = philox(P.key0, P.key1, make_uint4(j, g, 0u, P.tag | (ST_INIT << 4) | 1u));
      const float u[5] = {u01(w0.x), u01(w0.y), u01(w0.z), u01(w0.w), u01(w1.x)};
      if (P.init_kind == INIT_POINT || (P.init_kind == INIT_SHARING && g == 0)) {
#pragma unroll
        for (int d = 0; d < 5; ++d) s[d] = P.init_state[d];
        if (P.init_kind == INIT_SHARING) {
          // position uniform in the disc: r = R sqrt(u0), angle 2 pi u1
          const float r = P.init_radius * sqrtf(u[0]);
          float sn, cs;
          sincospif(fmaf(2.0f, u[1], -1.0f), &sn, &cs);  // angle 2 pi u1 - pi
          s[0] = P.init_state[0] - r * cs;
          s[1] = P.init_state[1] - r * sn;
        }
      } else {
#pragma unroll
        for (int d = 0; d < 5; ++d) s[d] = fmaf(P.init_hi[d] - P.init_lo[d], u[d], P.init_lo[d]);
      }
    }
    a.pv[i] = make_float4(s[0], s[1], s[2], s[3]);
    a.In[i] = s[4];
   }
  }
}

// ========================================================= frame preparation
// y = z - b into the interior of the zero-padded frame; the padding (2R+1
// pixels on each side, zeroed once at init) stands for "outside the image
// counts as background".
// y = z - b of one frame into its padded copy (rows offset by pad, pitch
// P.pitch), by the rows blockIdx.x, blockIdx.x + gridDim.x, ...  Frames
// with rows of whole float4 (and 16-byte aligned) are read four pixels per
// thread, several rows per block pass; the padded rows start off the 16-byte
// grid, so the stores stay scalar.
__device__ __forceinline__ void prep_rows(const float* __restrict__ z, float* __restrict__ yp, const TrackParams& P,
                                          int pad, float bg) {
  if ((P.W & 3) == 0 && (reinterpret_cast<uintptr_t>(z) & 15) == 0) {
    const int cols4 = P.W >> 2, nt = (int)blockDim.x;
    const int rpi = cols4 >= nt ? 1 : nt / cols4;  // rows per pass
    const int span = rpi == 1 ? nt : cols4;        // threads per row
    const int tr = (int)threadIdx.x / span, tc = (int)threadIdx.x - tr * span;
    if (tr < rpi)
      for (int v = (int)blockIdx.x * rpi + tr; v < P.H; v += (int)gridDim.x * rpi) {
        const float4* __restrict__ zr = reinterpret_cast<const float4*>(z + (long long)v * P.W);
        float* __restrict__ yr = yp + (long long)(v + pad) * P.pitch + pad;
        for (int c = tc; c < cols4; c += span) {
          const float4 q = __ldg(zr + c);
          yr[4 * c] = __fsub_rn(q.x, bg);
          yr[4 * c + 1] = __fsub_rn(q.y, bg);
          yr[4 * c + 2] = __fsub_rn(q.z, bg);
          yr[4 * c + 3] = __fsub_rn(q.w, bg);
        }
      }
    return;
  }
  for (int v = blockIdx.x; v < P.H; v += gridDim.x) {
    const float* __restrict__ zr = z + (long long)v * P.W;
    float* __restrict__ yr = yp + (long long)(v + pad) * P.pitch + pad;
    for (int u = threadIdx.x; u < P.W; u += blockDim.x) yr[u] = __fsub_rn(__ldg(zr + u), bg);
  }
}

__global__ void k_frame_prep(FrameArgs a) {
  grid_dep_wait();
  grid_dep_launch();
  if (blockIdx.x == 0 && blockIdx.y == 0)
    for (int i = threadIdx.x; i < a.nt; i += blockDim.x) a.frame_of[a.t0 + i] = a.share[i];
  const int tt = a.rep[blockIdx.y];
  const TrackParams& P = a.trk[a.t0 + tt];
  const float* __restrict__ z = a.frames[tt];
  float* __restrict__ yp = a.ypad + P.ypad_off;
  const int pad = 2 * a.R + 1;
  const float bg = P.bg;
  prep_rows(z, yp, P, pad, bg);
}

// Same, frame pointers from a device table indexed by the device-side step
// index: table[k * n_tracks + t] (k >= T_table is reported, not read).
__global__ void k_frame_prep_table(FrameTableArgs a) {
  grid_dep_wait();
  grid_dep_launch();
  const int t = blockIdx.y;
  const int k = a.ts[0].k;
  if (k >= a.T_table) {
    if (t == 0 && blockIdx.x == 0 && threadIdx.x == 0) set_error(a.ds, ERR_INDEX, 5u, (uint32_t)k, 0u);
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.frame_of[t] = t;
  const TrackParams& P = a.trk[t];
  const float* __restrict__ z = a.table[(long long)k * a.n_tracks + t];
  float* __restrict__ yp = a.ypad + P.ypad_off;
  const int pad = 2 * a.R + 1;
  const float bg = P.bg;
  prep_rows(z, yp, P, pad, bg);
}

// ================================================================ global step
// Per track: the master PE's reduction (Alg. 3 steps 9-10) and weight carry
// (step 8) for step k, then ring order (step 1) and exchange count (step 2)
// for step k+1.  G-sized; the exchange count is decided in FP64.
// log W^(m) = M + ln(Q 2^-40) in FP32: log2 Q from the leading-bit position
// and the top 24 bits of Q.
__device__ __forceinline__ float group_log_weight(float M, unsigned long long Q) {
  const int e = 63 - __clzll((long long)Q);
  const uint32_t top = e >= 23 ? (uint32_t)(Q >> (e - 23)) : (uint32_t)(Q << (23 - e));
  const float l2 = (float)(e - 23) + log2f((float)top);  // log2 Q (top is exact in FP32)
  return M + (l2 - 40.0f) * 0.693147182f;
}

// Scratch of the global step (shared memory of the CTA running it).
struct GlobalScratch {
  float f[32];
  int i[32];
  float red[32][6];
  unsigned long long w[32][2];
  float tot[6];
  double pe;
  int ring[MAX_G];
};

// The global step's inputs that the groups of the step do not write: the
// track's parameters and state, its ring, and the next step's ring and
// exchange offsets (drawn by the propagate kernel).  They can be read
// before the groups report.
template <int NT>
struct GlobalIn {
  static constexpr int GPT = (MAX_G + NT - 1) / NT;
  int G, Np, mode, topo, group_off, hist_off, k, nex_k;
  long long ghist_off;
  float cutoff, ex_ratio;
  double pe_k;
  int ring_m[GPT], rnext[GPT];
  uint32_t exo[GPT];
};

template <int NT>
__device__ __forceinline__ void global_load(const GlobalArgs& a, int t, GlobalIn<NT>& in) {
  const TrackParams* __restrict__ P = a.trk + t;
  in.G = P->G;
  in.Np = P->Np;
  in.mode = P->mode;
  in.topo = P->topology;
  in.group_off = P->group_off;
  in.hist_off = P->hist_off;
  in.ghist_off = P->ghist_off;
  in.cutoff = P->cutoff;
  in.ex_ratio = P->ex_ratio;
  const TrackState* __restrict__ T = a.ts + t;
  in.k = __ldcg(&T->k);
  in.nex_k = __ldcg(&T->n_ex);
  in.pe_k = __ldcg(&T->pe_eff);
  const int k1 = a.finalize ? in.k + 1 : 0;
  const int* __restrict__ ring = a.ring + in.group_off;
  const int* __restrict__ rnext_buf = a.ring_next + (size_t)(k1 & 1) * a.ring_stride + in.group_off;
  const uint32_t* __restrict__ exo_buf = a.exo_next + (size_t)(k1 & 1) * a.ring_stride + in.group_off;
#pragma unroll
  for (int i = 0; i < GlobalIn<NT>::GPT; ++i) {
    const int m = threadIdx.x + i * NT;
    in.ring_m[i] = m;
    in.rnext[i] = m;
    in.exo[i] = 0;
    if (m < in.G) {
      in.ring_m[i] = __ldcg(&ring[m]);
      in.rnext[i] = __ldcg(&rnext_buf[m]);
      in.exo[i] = __ldcg(&exo_buf[m]);
    }
  }
}

template <int NT>
__device__ __forceinline__ void global_step_core(const GlobalArgs& a, int t, GlobalScratch& sc,
                                                 const GlobalIn<NT>& in) {
  constexpr int NW = NT / 32;
  constexpr int GPT = GlobalIn<NT>::GPT;
  const int G = in.G, Np = in.Np, mode = in.mode, group_off = in.group_off, hist_off = in.hist_off;
  const long long ghist_off = in.ghist_off;
  const float cutoff = in.cutoff, ex_ratio = in.ex_ratio;
  TrackState* __restrict__ T = a.ts + t;
  const int k = in.k, nex_k = in.nex_k;
  const double pe_k = in.pe_k;
  GroupState* __restrict__ gs = a.gs + group_off;
  int* __restrict__ ring = a.ring + group_off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwa = G > NT ? NW : (G + 31) / 32;  // warps holding groups
  const int k1 = a.finalize ? k + 1 : 0;
  const int* ring_m = in.ring_m;
  const int* rnext = in.rnext;
  const uint32_t* exo = in.exo;

  // the groups' results of the step
  unsigned long long Q[GPT];
  float Mg[GPT], lam[GPT];
  int cy[GPT];
#pragma unroll
  for (int i = 0; i < GPT; ++i) {
    const int m = threadIdx.x + i * NT;
    Q[i] = 0;
    Mg[i] = 0.0f;
    cy[i] = 0;
    if (m < G) {
      Q[i] = __ldcg(&gs[m].Q);
      Mg[i] = __ldcg(&gs[m].M);
      if (a.finalize) cy[i] = __ldcg(&gs[m].carry_next);
    }
  }

  // S7 -> S8: Lambda'_m in FP32 (finalize), or 0 (prepare step 0)
  float mx = -INFINITY;
  int deg = 0;
#pragma unroll
  for (int i = 0; i < GPT; ++i) {
    const int m = threadIdx.x + i * NT;
    lam[i] = -INFINITY;
    if (m < G) {
      if (a.finalize) {
        lam[i] = Q[i] != 0 ? group_log_weight(Mg[i], Q[i]) : -INFINITY;
        deg += (Q[i] == 0) + (cy[i] ? 0 : 65536);  // degenerate and resampled groups (G < 2^15)
      } else {
        lam[i] = 0.0f;
      }
      mx = fmaxf(mx, lam[i]);
    }
  }
  mx = warp_max(mx);
  deg = __reduce_add_sync(0xffffffffu, deg);
  if (lane == 0) {
    sc.f[warp] = mx;
    sc.i[warp] = deg;
  }
  __syncthreads();
  mx = -INFINITY;
  deg = 0;
  for (int w = 0; w < nwa; ++w) {
    mx = fmaxf(mx, sc.f[w]);
    deg += sc.i[w];
  }
  const int res = deg >> 16;
  deg &= 0xffff;
  const bool all_degenerate = a.finalize && deg == G;
  if (all_degenerate) {  // every group lost its weight: restart from equal weights
#pragma unroll
    for (int i = 0; i < GPT; ++i) lam[i] = (threadIdx.x + i * NT < G) ? 0.0f : -INFINITY;
    mx = 0.0f;
  }
  // FP32 sum for log c; for Eq. 4 the FP64 weights w = e^(lam - max) in
  // (0, 1] and their squares, summed exactly as 2^-52 fixed-point integers
  // (at most G 2^52 < 2^63); the exchange count is decided in FP64 on both
  // sides.
  float wsum = 0.0f;
  unsigned long long iw = 0, iw2 = 0;
#pragma unroll
  for (int i = 0; i < GPT; ++i) {
    if (threadIdx.x + i * NT < G) {
      wsum += __expf(lam[i] - mx);
      const double w = exp((double)lam[i] - (double)mx);
      iw += __double2ull_rn(w * 4503599627370496.0);
      iw2 += __double2ull_rn(w * w * 4503599627370496.0);
    }
  }
  wsum = warp_sum(wsum);
  iw = warp_sum_u64(iw);
  iw2 = warp_sum_u64(iw2);
  if (lane == 0) {
    sc.red[warp][0] = wsum;
    sc.w[warp][0] = iw;
    sc.w[warp][1] = iw2;
  }
  // ring order of step k1 (Sec. IV-B), drawn one step ahead; for the
  // hypercube each group's partner
  const int topo = in.topo;
  const bool shuffled = k1 >= 1 && G > 1 && (mode == MODE_ARNA || topo == TOPO_HYPERCUBE);
#pragma unroll
  for (int i = 0; i < GPT; ++i) {
    const int m = threadIdx.x + i * NT;
    if (m < G) sc.ring[m] = shuffled ? rnext[i] : m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float x = 0.0f;
    for (int w = 0; w < nwa; ++w) x += sc.red[w][0];
    sc.tot[0] = x;
  }
  if (threadIdx.x == (NW > 1 ? 32 : 7)) {
    unsigned long long s1 = 0, s2 = 0;
    for (int w = 0; w < nwa; ++w) {
      s1 += sc.w[w][0];
      s2 += sc.w[w][1];
    }
    const double sw = (double)s1, sw2 = (double)s2;
    const double pe = sw * sw / sw2 * 2.220446049250313e-16;  // Eq. 4 for the next step (scales 2^-52)
    // exchange count for step k1 (Eq. 3 with the Sec. V-A cut-off)
    int nex = 0;
    if (k1 >= 1 && G > 1) {
      double rho;
      if (mode == MODE_ARNA) {
        if (!(pe < (double)cutoff * (double)G)) {
          rho = 0.0;
        } else {
          rho = 0.5 - 0.5 * (pe - 1.0) / (double)(G - 1);
          rho = fmin(fmax(rho, 0.0), 0.5);
        }
      } else {
        rho = fmin(fmax((double)ex_ratio, 0.0), 1.0);
      }
      nex = (int)floor(rho * (double)Np);
    }
    sc.pe = pe;
    sc.i[0] = nex;
  }
  __syncthreads();
  const float lse = mx + logf(sc.tot[0]);  // LSE of the carried weights = log c_k
  const double pe = sc.pe;
  const int nex = sc.i[0];
  const float log_np = logf((float)Np);

  if (a.finalize) {
    // history fields the next step overwrites: ring, exchange count, PE_eff
    const int hslot = k % a.history;
#pragma unroll
    for (int i = 0; i < GPT; ++i) {
      const int m = threadIdx.x + i * NT;
      if (m < G) a.ghist[ghist_off + (long long)hslot * G + m].ring = ring_m[i];
    }
    if (threadIdx.x == 0) {
      HistRec& h = a.hist[hist_off + hslot];
      h.step = k;
      h.n_ex = nex_k;
      h.pe_eff = pe_k;
    }
  }
#pragma unroll
  for (int i = 0; i < GPT; ++i) {
    const int m = threadIdx.x + i * NT;
    if (m < G) {
      int rm = sc.ring[m];
#ifdef PF_DEBUG
      rm = (int)PF_DBG_INDEX(a.ds, rm, G, 301u);
#endif
      ring[m] = rm;
      if (topo == TOPO_HYPERCUBE)
        gs[m].pred = rm;  // mutual exchange with the partner
      else
        gs[rm].pred = sc.ring[m == 0 ? G - 1 : m - 1];
      gs[m].exo = nex > 0 ? exo[i] : 0u;
      gs[m].lambda = lam[i];
      // S4: a resampled group's particles weigh W_m / Np, a group that kept
      // its particles passes their own log-weights on (log w~ - LSE)
      gs[m].off = cy[i] ? -lse : lam[i] - log_np - lse;
      // the resampler's decision of step k, read by step k1's propagation
      gs[m].carry = cy[i];
      if (!a.finalize) gs[m].carry_next = 0;
    }
  }
  if (threadIdx.x == 0) {
    T->n_ex = nex;
    T->pe_eff = pe;
    T->deg_k = a.finalize ? deg : 0;
    T->res_k = a.finalize ? res : 0;
    T->lse_k = lse;
    if (!a.finalize) T->fin_k = -1;
    if (!a.keep_k) T->k = k1;
  }
}

// The global step of track t by one CTA of NT threads, each thread owning
// groups m = threadIdx.x + i NT: what the next step needs (group weights
// carried as offsets, Eq. 3 / Eq. 4 exchange count, ring order and
// exchange offsets, step index) plus the history fields that it is about to
// overwrite.  The estimate, log c, log Z and the rest of the history follow
// in finish_step, off the critical path.  finalize = 0 prepares step 0.
// Per-group inputs are read through L2 (written by other CTAs of the same
// launch when this runs as the resampler's tail).  Every input is read
// before the first store (so no load waits behind a store that might alias
// it).
template <int NT>
__device__ __forceinline__ void global_step(const GlobalArgs& a, int t, GlobalScratch& sc) {
  GlobalIn<NT> in;
  global_load<NT>(a, t, in);
  global_step_core<NT>(a, t, sc, in);
}

// global_step out of line, for the resampler (it runs on one CTA of the
// launch, and inlined twice it would crowd the resampler's own registers).
template <int NT>
__device__ __noinline__ void global_step_call(const GlobalArgs& a, int t, GlobalScratch& sc) {
  global_step<NT>(a, t, sc);
}

// The rest of the global step of the track's last finished step kd = k - 1
// (Alg. 3 steps 9-10 and the history): global estimate from the group
// estimates and carried weights, log c = the carried weights' LSE, log Z,
// per-group history.  Run once per step (guarded by fin_k) by a leading
// block of the next propagate launch, or by k_finish before the host reads
// the statistics; one CTA of NT threads.
template <int NT>
__device__ void finish_step(const GlobalArgs& a, int t, GlobalScratch& sc) {
  constexpr int NW = NT / 32;
  constexpr int GPT = (MAX_G + NT - 1) / NT;
  const TrackParams* __restrict__ P = a.trk + t;
  TrackState* __restrict__ T = a.ts + t;
  const int kd = __ldcg(&T->k) - 1;
  if (kd < 0 || __ldcg(&T->fin_k) >= kd) return;  // uniform over the CTA
  const int G = P->G, group_off = P->group_off, hist_off = P->hist_off;
  const long long ghist_off = P->ghist_off;
  const int deg = __ldcg(&T->deg_k);
  const float lse = __ldcg(&T->lse_k);
  const double logZ_prev = __ldcg(&T->log_Z);
  const int flags = __ldcg(&T->flags);
  const GroupState* __restrict__ gs = a.gs + group_off;
  const bool all_degenerate = deg == G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwa = G > NT ? NW : (G + 31) / 32;

  float lam[GPT], xs[GPT][5], ess[GPT];
  float mx = -INFINITY;
#pragma unroll
  for (int i = 0; i < GPT; ++i) {
    const int m = threadIdx.x + i * NT;
    lam[i] = -INFINITY;
    ess[i] = 0.0f;
#pragma unroll
    for (int q = 0; q < 5; ++q) xs[i][q] = 0.0f;
    if (m < G) {
      lam[i] = __ldcg(&gs[m].lambda);
#pragma unroll
      for (int q = 0; q < 5; ++q) xs[i][q] = __ldcg(&gs[m].xs[q]);
      ess[i] = __ldcg(&gs[m].ess);
      mx = fmaxf(mx, lam[i]);
    }
  }
  mx = warp_max(mx);
  if (lane == 0) sc.f[warp] = mx;
  __syncthreads();
  mx = -INFINITY;
  for (int w = 0; w < nwa; ++w) mx = fmaxf(mx, sc.f[w]);
  float acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < GPT; ++i) {
    if (threadIdx.x + i * NT < G) {
      const float wf = __expf(lam[i] - mx);
      acc[0] += wf;
#pragma unroll
      for (int q = 0; q < 5; ++q) acc[1 + q] = fmaf(wf, xs[i][q], acc[1 + q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) acc[q] = warp_sum(acc[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 6; ++q) sc.red[warp][q] = acc[q];
  __syncthreads();
  if (threadIdx.x < 6) {
    float x = 0.0f;
    for (int w = 0; w < nwa; ++w) x += sc.red[w][threadIdx.x];
    sc.tot[threadIdx.x] = x;
  }
  __syncthreads();
  const int hslot = kd % a.history;
#pragma unroll
  for (int i = 0; i < GPT; ++i) {
    const int m = threadIdx.x + i * NT;
    if (m < G) {
      GroupHist& gh = a.ghist[ghist_off + (long long)hslot * G + m];
      gh.logW = all_degenerate ? -INFINITY : lam[i];
#pragma unroll
      for (int q = 0; q < 5; ++q) gh.xs[q] = xs[i][q];
      gh.ess = ess[i];
    }
  }
  if (threadIdx.x == 0) {
    const double logc = all_degenerate ? -INFINITY : (double)lse;
    const double logZ = logZ_prev + logc;
    float xq[5];
    for (int q = 0; q < 5; ++q) xq[q] = all_degenerate ? NAN : sc.tot[1 + q] / sc.tot[0];
    HistRec& h = a.hist[hist_off + hslot];
    for (int q = 0; q < 5; ++q) h.xhat[q] = xq[q];
    h.log_c = logc;
    h.log_Z = logZ;
    h.degenerate = deg;
    h.resampled = __ldcg(&T->res_k);
    T->log_c = logc;
    T->log_Z = logZ;
    for (int q = 0; q < 5; ++q) T->xhat[q] = xq[q];
    T->degenerate = deg;
    T->flags = flags | (all_degenerate ? 1 : 0);
    T->steps_done = kd + 1;
    T->fin_k = kd;
  }
}

// Per track: the master PE's reduction (Alg. 3 steps 9-10) and weight carry
// (step 8) for step k, then ring order (step 1) and exchange count (step 2)
// for step k+1 (global_step; finalize = 0 prepares step 0).  During the run
// the same step runs as the tail of the resampler.
__global__ void __launch_bounds__(GL_THREADS) k_global(GlobalArgs a) {
  __shared__ GlobalScratch sc;
  global_step<GL_THREADS>(a, blockIdx.x, sc);
}

// finish_step for every track (one CTA each), before the host reads the
// statistics of the last step.
__global__ void __launch_bounds__(K1_THREADS) k_finish(GlobalArgs a) {
  __shared__ GlobalScratch sc;
  finish_step<K1_THREADS>(a, blockIdx.x, sc);
}

// k_finish, then the track's x^ and log Z stored straight into the caller's
// page-locked host buffers (their device addresses; either may be null), so
// that reading the estimate back takes no copy on the stream.  It may be
// launched while the resampler drains (programmatic dependent launch) and
// waits for it before reading anything.
struct FinishOutArgs {
  GlobalArgs g;
  float* xhat;
  double* logZ;
};

__global__ void __launch_bounds__(K1_THREADS) k_finish_out(FinishOutArgs a) {
  __shared__ GlobalScratch sc;
  grid_dep_wait();
  finish_step<K1_THREADS>(a.g, blockIdx.x, sc);
  if (threadIdx.x == 0) {  // the thread that wrote the track state, if finish_step ran here
    const TrackState* T = a.g.ts + blockIdx.x;
    if (a.xhat)
      for (int q = 0; q < 5; ++q) a.xhat[blockIdx.x * 5 + q] = __ldcg(&T->xhat[q]);
    if (a.logZ) a.logZ[blockIdx.x] = __ldcg(&T->log_Z);
  }
}

// ============================================================ propagate + weight
// Fisher-Yates ring order of step k (Sec. IV-B, Alg. 3 step 1) for one
// track, by one warp: the bounded draws r_j in [0, j] in parallel, the
// descending swaps by lane 0 in shared memory.
__device__ void ring_for_step(const TrackParams& P, int track, uint32_t k, int* __restrict__ out, int* __restrict__ sh,
                              DevState* ds) {
  const int lane = threadIdx.x & 31;
  const int G = P.G;
  for (int p = lane; p < G; p += 32) {
    uint32_t r = 0;
    if (p >= 1 && !draw_bounded(P.key0, P.key1, P.tag, ST_RING, (uint32_t)p, k, (uint32_t)p + 1u, r))
      set_error(ds, ERR_DRAW, 1u, (uint32_t)track, (uint32_t)p);
    sh[p] = (int)r;           // r_j, turned into the permutation below
    out[p] = p;
  }
  __syncwarp();
  if (lane == 0) {
    for (int j = G - 1; j >= 1; --j) {
      const int r = sh[j];
      const int tmp = out[j];
      out[j] = out[r];
      out[r] = tmp;
    }
  }
  __syncwarp();
}

// The exchange pattern of step k for the other topologies (Sec. VI), by one
// warp, into out[0 .. G) (not inlined: leading blocks only, and inlining it
// slowed the propagate kernel's tiles by ~1 us through code size): TOPO_NODE_RING (ARNA): nodes of node_groups
// consecutive groups, the ring visiting the nodes in a Fisher-Yates order
// (draw j from RING call 1, index j) and each node's groups in a
// Fisher-Yates order (draw j from RING call 2, index n node_groups + j);
// TOPO_HYPERCUBE: out[g] = g's partner g xor 2^d (g itself when that is
// >= G), d = (k - 1) mod D (RNA) or drawn from RING call 3, index 0 (ARNA).
__device__ __noinline__ void topology_for_step(const TrackParams& P, int track, uint32_t k, int* __restrict__ out,
                                  int* __restrict__ sh, DevState* ds) {
  const int lane = threadIdx.x & 31;
  const int G = P.G;
  if (P.topology == TOPO_HYPERCUBE) {
    uint32_t d = 0;
    if (P.mode == MODE_ARNA) {
      if (!draw_bounded(P.key0, P.key1, P.tag | 3u, ST_RING, 0u, k, (uint32_t)P.hyper_dims, d))
        set_error(ds, ERR_DRAW, 3u, (uint32_t)track, 0u);
    } else {
      d = (k - 1u) % (uint32_t)P.hyper_dims;
    }
    for (int g = lane; g < G; g += 32) {
      const int p = g ^ (1 << d);
      out[g] = p < G ? p : g;
    }
    __syncwarp();
    return;
  }
  // node-aware ring.  Scratch: node draws (NN), node order (NN), member
  // draws by group (G), one node's member order (B): at most 3 G + 1 ints.
  const int B = P.node_groups < G ? P.node_groups : G, NN = (G + B - 1) / B;
  int* rn = sh;
  int* nodes = sh + NN;
  int* rm = sh + 2 * NN;
  int* mem = rm + G;
  for (int j = lane; j < NN; j += 32) {
    uint32_t r = 0;
    if (j >= 1 && !draw_bounded(P.key0, P.key1, P.tag | 1u, ST_RING, (uint32_t)j, k, (uint32_t)j + 1u, r))
      set_error(ds, ERR_DRAW, 4u, (uint32_t)track, (uint32_t)j);
    rn[j] = (int)r;
  }
  for (int gi = lane; gi < G; gi += 32) {
    const int j = gi % B;  // position within its node
    uint32_t r = 0;
    if (j >= 1 && !draw_bounded(P.key0, P.key1, P.tag | 2u, ST_RING, (uint32_t)gi, k, (uint32_t)j + 1u, r))
      set_error(ds, ERR_DRAW, 5u, (uint32_t)track, (uint32_t)gi);
    rm[gi] = (int)r;
  }
  __syncwarp();
  if (lane == 0) {
    for (int n = 0; n < NN; ++n) nodes[n] = n;
    for (int j = NN - 1; j >= 1; --j) {
      const int r = rn[j], t = nodes[j];
      nodes[j] = nodes[r];
      nodes[r] = t;
    }
    int pos = 0;
    for (int q = 0; q < NN; ++q) {
      const int base = nodes[q] * B, sz = G - base < B ? G - base : B;
      for (int i = 0; i < sz; ++i) mem[i] = base + i;
      for (int j = sz - 1; j >= 1; --j) {
        const int r = rm[base + j], t = mem[j];
        mem[j] = mem[r];
        mem[r] = t;
      }
      for (int i = 0; i < sz; ++i) out[pos++] = mem[i];
    }
  }
  __syncwarp();
}

// ---- TMA / mbarrier helpers (inline PTX) ---------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity`, for at most MBAR_WAIT_NS; false if it did not
// complete (a copy that never lands ends the wait instead of the kernel).
constexpr unsigned long long MBAR_WAIT_NS = 200000000ull;  // 0.2 s
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u && global_ns() - t0 > MBAR_WAIT_NS) return false;
  }
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_2d(float* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Systematic send sets (Sec. III-C): slot j of group g takes the
// predecessor's slot src_j (true) when j is the t-th send slot
// floor((t Np + o_r) / N_ex) of the receiver, src_j = floor((t Np + o_s) /
// N_ex) being the sender's t-th; else it keeps its own slot j (false).  The
// group's exchange offsets o_r (receiver) and o_s (sender) are hoisted out
// of the particle loop.
__device__ __forceinline__ bool exchange_from_pred(int j, int Np, int nex, uint32_t o_r, uint32_t o_s,
                                                   unsigned long long mNp, int& src_j) {
  src_j = j;
  if (nex <= 0) return false;
  if ((unsigned long long)Np * (unsigned long long)(nex + 1) < (1ull << 32)) {
    const uint32_t jn = (uint32_t)j * (uint32_t)nex;
    const uint32_t t = jn <= o_r ? 0u : fastdiv(jn - o_r + (uint32_t)Np - 1u, mNp);
    if (t < (uint32_t)nex && t * (uint32_t)Np + o_r < jn + (uint32_t)nex) {
      src_j = (int)((t * (uint32_t)Np + o_s) / (uint32_t)nex);
      return true;
    }
    return false;
  }
  const long long num = (long long)j * nex - o_r;
  const long long t = num <= 0 ? 0 : (num + Np - 1) / Np;
  if (t < nex && t * Np + o_r < (long long)(j + 1) * nex) {
    src_j = (int)((t * Np + o_s) / nex);
    return true;
  }
  return false;
}

// Keyed send sets (Sec. III-C, "randomly selects"): group g sends slots
// pi_g(t), t < N_ex, of a keyed permutation of [0, Np): a four-round Feistel
// network (Luby-Rackoff) on b = ceil(log2 Np) bits, the high half L of
// floor(b/2) bits and the low half R of the rest; a round maps (L, R) to
// (R, L xor (F(R xor key_i) mod 2^|L|)), so the halves trade places and
// sizes; values >= Np walk on through the network until they land in
// [0, Np) (cycle walking, Black-Rogaway), which ends within 2^b rounds of
// the walk since the network permutes [0, 2^b).  F: h = x * 0x9E3779B1,
// h ^= h >> 16, h *= 0x7FEB352D, h ^= h >> 15.
__device__ __forceinline__ uint32_t feistel_f(uint32_t x) {
  uint32_t h = x * 0x9E3779B1u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  return h ^ (h >> 15);
}

__device__ __forceinline__ uint32_t send_perm(uint32_t t, uint32_t n, int b, uint4 key) {
  const uint32_t kk[4] = {key.x, key.y, key.z, key.w};
  uint32_t x = t;
  do {
    int sl = b >> 1, sr = b - sl;
    uint32_t L = x >> sr, R = x & ((1u << sr) - 1u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t nr = L ^ (feistel_f(R ^ kk[i]) & ((1u << sl) - 1u));
      L = R;
      R = nr;
      const int s = sl;
      sl = sr;
      sr = s;
    }
    x = (L << sr) | R;
  } while (x >= n);
  return x;
}

__device__ __forceinline__ uint32_t send_perm_inv(uint32_t j, uint32_t n, int b, uint4 key) {
  const uint32_t kk[4] = {key.x, key.y, key.z, key.w};
  uint32_t x = j;
  do {
    int sl = b >> 1, sr = b - sl;
    uint32_t L = x >> sr, R = x & ((1u << sr) - 1u);
#pragma unroll
    for (int i = 3; i >= 0; --i) {
      const uint32_t nl = R ^ (feistel_f(L ^ kk[i]) & ((1u << sr) - 1u));
      R = L;
      L = nl;
      const int s = sl;
      sl = sr;
      sr = s;
    }
    x = (L << sr) | R;
  } while (x >= n);
  return x;
}

// Slot j of the receiver takes the predecessor's slot pi_s(t) when
// t = pi_r^-1(j) < N_ex (keys k_r of the receiver, k_s of the sender).
__device__ __forceinline__ bool exchange_keyed(int j, int Np, int nex, int b, uint4 k_r, uint4 k_s, int& src_j) {
  const uint32_t t = send_perm_inv((uint32_t)j, (uint32_t)Np, b, k_r);
  if (t < (uint32_t)nex) {
    src_j = (int)send_perm(t, (uint32_t)Np, b, k_s);
    return true;
  }
  src_j = j;
  return false;
}

// Hint: bring [p, p + bytes) into L2 (one bulk prefetch; the range is
// widened to 16-byte boundaries, which stay inside the workspace).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const unsigned long long a0 = (unsigned long long)p & ~15ull;
  const unsigned long long a1 = ((unsigned long long)p + bytes + 15ull) & ~15ull;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
}

// The previous step's ancestors, states and intensities of a tile's slot
// range: without weight degeneracy the parents of slots j.. lie near j.
__device__ __forceinline__ void prefetch_tile(const K1Args& a, int4 td, int k, const float4* pv_prev,
                                              const float* I_prev) {
  const TrackParams& P = a.trk[td.x];
  const long long i0 = P.part_off + (long long)td.y * P.Np + td.z;
  if (k > 0) prefetch_l2(a.anc + ((k + 1) & 1) * a.anc_stride + i0, sizeof(uint32_t) * (size_t)td.w);
  prefetch_l2(pv_prev + i0, sizeof(float4) * (size_t)td.w);
  prefetch_l2(I_prev + i0, sizeof(float) * (size_t)td.w);
}

// The five process-noise normals of slot j of group g at step k (Alg. 1
// step P): Philox stream PROP, calls 0 and 1, Box-Muller on word pairs.
// RK: the track's precomputed round keys (parameters in the constant bank).
template <bool RK>
__device__ __forceinline__ void prop_noise(const TrackParams& P, int j, int g, int k, float (&e)[5]) {
  uint4 w0 = make_uint4(j, g, k, P.tag | (ST_PROP << 4) | 0u);
  uint4 w1 = make_uint4(j, g, k, P.tag | (ST_PROP << 4) | 1u);
  if constexpr (RK)
    philox2_rk(P.rk, w0, w1);
  else
    philox2(P.key0, P.key1, w0, w1);
  float e5;
  box_muller_fast(w0.x, w0.y, e[0], e[1]);
  box_muller_fast(w0.z, w0.w, e[2], e[3]);
  box_muller_fast(w1.x, w1.y, e[4], e5);
}

// Ready-queue entries of the fused step: task kind << RQ_KIND_SHIFT | index.
constexpr uint32_t RQ_KIND_SHIFT = 28;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Fused step tasks and scheduling (defined with the resampler below).
__device__ __noinline__ void fused_task_a(const K1Args& a, int k, int ci, unsigned char* smem);
__device__ __noinline__ void fused_task_b(const K1Args& a, int k, int ci, unsigned char* smem);
__device__ __noinline__ void fused_group_tiles_done(const K1Args& a, int k, int gi);
__device__ __noinline__ int rq_try_claim(const K1Args& a, int par);
__device__ __noinline__ int rq_entry(const K1Args& a, int par, unsigned pos);
__device__ __noinline__ int rq_wait_claim(const K1Args& a, int par);
__device__ __forceinline__ bool step_failed(const DevState* ds);

// Shared memory of the fused step: the staged frame box of a P task, or the
// prefixes and ancestor window of a B task, or the global step's scratch.
constexpr size_t FUSED_SMEM = sizeof(unsigned long long) * pad8(RS_CHUNK) + sizeof(uint32_t) * pad8(2 * RS_CHUNK);
constexpr size_t ROI_SMEM = sizeof(float) * 2 * (ROI_FLOATS + 4);
static_assert(ROI_SMEM <= FUSED_SMEM && sizeof(GlobalScratch) <= FUSED_SMEM, "fused step shared memory");

// Propagate + weight: tiles of K1_TILE = K1_PPT x K1_THREADS slots of one
// group, K1_PPT particles per thread.  Each tile stages the bounding box of
// its particles' patches (at most ROI_W x ROI_ROWS floats) in shared memory
// by TMA; tiles whose patches do not fit read the frame through L1.
// Leading blocks draw the next step's rings and exchange offsets and finish
// the previous step.
// SINGLE: one track, whose parameters come from the kernel's constant
// parameter block (a.p0) instead of global memory.
// FUSED: the whole step in this launch -- the tiles are the P tasks, taken
// between the resampling tasks A and B as those become ready (see "fused
// step" below); the step index advances when the last CTA leaves.
template <int R, bool SINGLE, bool VARIANTS, bool FUSED>
__global__ void __launch_bounds__(K1_THREADS, K1_MIN_BLOCKS) k_propagate_weight(const __grid_constant__ K1Args a) {
  constexpr int D = 2 * R + 1;
  constexpr int PAD = 2 * R + 1;
  constexpr int NW = K1_THREADS / 32;
  // the staged box (TMA target) and a copy shifted left by one float, so that
  // any patch row starts on an 8-byte boundary in one of the two (pairwise
  // loads); 4 spare floats cover the last pair of the last row.  The fused
  // step keeps it in dynamic shared memory, shared with the other tasks.
  __shared__ __align__(128) float s_roi_static[FUSED ? 1 : 2][FUSED ? 4 : ROI_FLOATS + 4];
  extern __shared__ __align__(128) unsigned char s_dyn[];
  float (*s_roi)[ROI_FLOATS + 4] = FUSED ? reinterpret_cast<float (*)[ROI_FLOATS + 4]>(s_dyn)
                                         : reinterpret_cast<float (*)[ROI_FLOATS + 4]>(&s_roi_static[0][0]);
  __shared__ int s_next[2];  // next tile, by iteration parity
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ float s_red[NW][8];
  __shared__ int s_box[NW][4];
  __shared__ int s_key[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int stride = (int)gridDim.x - a.n_ring_blocks;
  int tile = (int)blockIdx.x - a.n_ring_blocks;
  grid_dep_wait();
  grid_dep_launch();
  const int k = a.ts[0].k;
  const float4* __restrict__ pv_prev = (k & 1) ? a.pv0 : a.pv1;
  const float* __restrict__ I_prev = (k & 1) ? a.I0 : a.I1;
  float4* __restrict__ pv_cur = (k & 1) ? a.pv1 : a.pv0;
  float* __restrict__ I_cur = (k & 1) ? a.I1 : a.I0;
  if ((int)blockIdx.x < a.n_ring_blocks) {
    // Leading blocks, off the critical path: per track the next step's
    // exchange offsets o_g (Sec. III-C send sets) and ARNA ring order (they
    // depend only on the seed and the step index), then the previous step's
    // estimate, log c, log Z and history (finish_step).
    static_assert(sizeof(GlobalScratch) <= ROI_SMEM, "the leading blocks' scratch lives in s_roi");
    // the fused step's counters of the next step (this launch uses parity
    // k & 1; the previous launch, which used the other parity, has ended)
    if (a.sync) {
      const FusedSync fs{a.ring_stride};
      const int par1 = (k + 1) & 1;
      for (int i = blockIdx.x * K1_THREADS + threadIdx.x; i < a.ring_stride; i += a.n_ring_blocks * K1_THREADS) {
        a.sync[fs.pdone(par1, i)] = 0u;
        a.sync[fs.adone(par1, i)] = 0u;
      }
      unsigned* q1 = a.rq + (size_t)par1 * 2 * a.n_chunks;
      for (int i = blockIdx.x * K1_THREADS + threadIdx.x; i < 2 * a.n_chunks; i += a.n_ring_blocks * K1_THREADS)
        q1[i] = 0u;
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.sync[fs.tile_ctr(par1)] = 0u;
        a.sync[fs.exit_ctr(par1)] = 0u;
        a.sync[fs.ring_done(par1)] = 0u;
        a.sync[fs.rq_head(par1)] = 0u;
        a.sync[fs.rq_tail(par1)] = 0u;
      }
    }
    const GlobalArgs ga{a.trk, a.ts, a.grp, nullptr, a.ring_next, a.ring_stride, a.exo_next, a.hist, a.ghist,
                        a.history, 1, a.ds};
    int* perm = reinterpret_cast<int*>(&s_roi[0][0]);
    int* rr = perm + RING_SMEM_G;
    for (int t = blockIdx.x; t < a.n_tracks; t += a.n_ring_blocks) {
      const TrackParams& P = a.trk[t];
      uint32_t* exo_out = a.exo_next + (size_t)((k + 1) & 1) * a.ring_stride + P.group_off;
      uint4* keys_out = a.keys_next + (size_t)((k + 1) & 1) * a.ring_stride + P.group_off;
      for (int m = threadIdx.x; m < P.G; m += K1_THREADS) {
        uint32_t o = 0;
        if (P.G > 1 && !draw_bounded(P.key0, P.key1, P.tag, ST_EXCH, (uint32_t)m, (uint32_t)(k + 1), (uint32_t)P.Np, o))
          set_error(a.ds, ERR_DRAW, 2u, (uint32_t)t, (uint32_t)m);
        exo_out[m] = o;
        // keyed send sets: the permutation's round keys (EXCH stream, call 1)
        if (P.send_rule == 1 && P.G > 1)
          keys_out[m] = philox(P.key0, P.key1, make_uint4((uint32_t)m, 0u, (uint32_t)(k + 1), P.tag | (ST_EXCH << 4) | 1u));
      }
      if (warp == 0 && P.G > 1 && P.G <= RING_SMEM_G &&
          (P.topology == TOPO_HYPERCUBE || (P.mode == MODE_ARNA && P.topology == TOPO_NODE_RING))) {
        topology_for_step(P, t, (uint32_t)(k + 1), perm, rr, a.ds);
        for (int p = lane; p < P.G; p += 32)
          a.ring_next[(size_t)((k + 1) & 1) * a.ring_stride + P.group_off + p] = perm[p];
      } else if (warp == 0 && P.mode == MODE_ARNA && P.G > 1 && P.G <= RING_SMEM_G) {
        ring_for_step(P, t, (uint32_t)(k + 1), perm, rr, a.ds);
        for (int p = lane; p < P.G; p += 32)
          a.ring_next[(size_t)((k + 1) & 1) * a.ring_stride + P.group_off + p] = perm[p];
      }
      __syncthreads();  // s_roi free for the scratch
      finish_step<K1_THREADS>(ga, t, *reinterpret_cast<GlobalScratch*>(&s_roi[0][0]));
      __syncthreads();
    }
    if constexpr (!FUSED) return;
  }
  __shared__ int s_last;
  if (FUSED && (int)blockIdx.x < a.n_ring_blocks) {
    // the group finalisations of this step wait for the leading blocks
    // (they read the previous step's group state, which those overwrite)
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&a.sync[FusedSync{a.ring_stride}.ring_done(k & 1)], 1u);
    }
  }
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    fence_proxy_async();
    if (!FUSED && tile < a.n_tiles) prefetch_tile(a, a.tiles[tile], k, pv_prev, I_prev);
  }
  __syncthreads();
  uint32_t phase = 0;
  // SINGLE: the track's exchange count for the whole launch
  const int nex1 = SINGLE && k > 0 ? a.ts[0].n_ex : 0;

  auto run_tile = [&](const TrackParams& P, const int4 td) {
    const int g = td.y, Np = P.Np;
    // the padded frame to read: the track's own, or the copy of a track
    // given the same frame this step
    const int ft = SINGLE ? 0 : (a.frame_of ? __ldg(&a.frame_of[td.x]) : td.x);
    const long long ypad_off = (SINGLE || ft == td.x) ? P.ypad_off : a.trk[ft].ypad_off;
    const GroupState* __restrict__ gs = a.grp + P.group_off;
    const int nex = SINGLE ? nex1 : (k > 0 ? a.ts[td.x].n_ex : 0);
    // the group's exchange partners and weight offsets, once per tile
    const float off_g = gs[g].off;
    uint32_t o_r = 0, o_s = 0;
    int sg = g;
    float off_s = off_g;
    if (nex > 0) {
      o_r = gs[g].exo;
      sg = gs[g].pred;
#ifdef PF_DEBUG
      sg = (int)PF_DBG_INDEX(a.ds, sg, P.G, 105u);
#endif
      o_s = gs[sg].exo;
      off_s = gs[sg].off;
    }
    // keyed send sets: the receiver's and the sender's permutation keys
    const bool keyed = VARIANTS && P.send_rule == 1 && nex > 0;
    uint4 key_r = make_uint4(0u, 0u, 0u, 0u), key_s = key_r;
    if (keyed) {
      const uint4* kb = a.keys_next + (size_t)(k & 1) * a.ring_stride + P.group_off;
      key_r = kb[g];
      key_s = kb[sg];
    }
    // bit 0: this group kept its particles at the last step, bit 1: the
    // sending group did; their particles pass their own log-weights on
    const int cmask = (VARIANTS && k > 0) ? (gs[g].carry | (gs[sg].carry << 1)) : 0;
    const uint32_t n_track = (uint32_t)(P.G * Np);
    const uint32_t* __restrict__ anc_t = a.anc + ((k + 1) & 1) * a.anc_stride + P.part_off;  // step k - 1's
    const float4* __restrict__ pvp_t = pv_prev + P.part_off;
    const float* __restrict__ Ip_t = I_prev + P.part_off;
    float4* __restrict__ pvc_t = pv_cur + P.part_off;
    float* __restrict__ Ic_t = I_cur + P.part_off;
    float* __restrict__ lw_t = ((VARIANTS && (k & 1)) ? a.lw1 : a.lw) + P.part_off;
    uint32_t* __restrict__ par_t =
        P.record ? a.parent + P.parent_off + (long long)(k % a.history) * (long long)n_track : nullptr;
    float4 s[K1_PPT];
    float I[K1_PPT];
    bool from_pred[K1_PPT];
    int pu[K1_PPT], pv[K1_PPT];
    int umin = INT_MAX, umax = INT_MIN, vmin = INT_MAX, vmax = INT_MIN;
#pragma unroll
    for (int q = 0; q < K1_PPT; ++q) {
      const int jj = threadIdx.x + q * K1_THREADS;
      const bool active = jj < td.w;
      const int j = td.z + jj;
      const int il = g * Np + j;
      s[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      I[q] = 0.0f;
      from_pred[q] = false;
      if (active) {
        int sj;
        from_pred[q] = keyed ? exchange_keyed(j, Np, nex, P.perm_bits, key_r, key_s, sj)
                             : exchange_from_pred(j, Np, nex, o_r, o_s, P.m_Np, sj);
        uint32_t src = (uint32_t)((from_pred[q] ? sg : g) * Np + sj);
#ifdef PF_DEBUG
        src = (uint32_t)PF_DBG_INDEX(a.ds, src, n_track, 101u);
        PF_DBG_INDEX(a.ds, il, n_track, 102u);
#endif
        const uint32_t par = (k == 0) ? src : anc_t[src];
        if (par >= n_track) {
          set_error(a.ds, ERR_INDEX, 1u, (uint32_t)tile, par);
        } else {
          s[q] = pvp_t[par];
          I[q] = Ip_t[par];
          // A group that kept its particles passes their own log-weights on:
          // the particle's weight offset is parked in its output slot until
          // the likelihood is added (no register held across the patch sum).
          if (VARIANTS && ((cmask >> (from_pred[q] ? 1 : 0)) & 1))
            lw_t[il] = (from_pred[q] ? off_s : off_g) + ((k & 1) ? a.lw : a.lw1)[P.part_off + par];
        }
        if (k > 0) {
          // Alg. 1 step P: nearly constant velocity, unit frame interval
          float e[5];
          prop_noise<SINGLE>(P, j, g, k, e);
          s[q].x = fmaf(P.spos, e[0], s[q].x + s[q].z);
          s[q].y = fmaf(P.spos, e[1], s[q].y + s[q].w);
          s[q].z = fmaf(P.sv, e[2], s[q].z);
          s[q].w = fmaf(P.sv, e[3], s[q].w);
          I[q] = fmaf(P.sI, e[4], I[q]);
        }
        pvc_t[il] = s[q];
        Ic_t[il] = I[q];
        if (par_t) par_t[il] = par;
        // patch corner in padded-frame coordinates (centre clamped so that a
        // patch wholly off the frame reads the zero border)
        pu[q] = (int)fminf(fmaxf(floorf(s[q].x + 0.5f), -(float)(R + 1)), (float)(P.W + R)) - R + PAD;
        pv[q] = (int)fminf(fmaxf(floorf(s[q].y + 0.5f), -(float)(R + 1)), (float)(P.H + R)) - R + PAD;
        umin = min(umin, pu[q]);
        umax = max(umax, pu[q]);
        vmin = min(vmin, pv[q]);
        vmax = max(vmax, pv[q]);
      }
    }

    // tile bounding box of the patches
    umin = __reduce_min_sync(0xffffffffu, umin);
    umax = __reduce_max_sync(0xffffffffu, umax);
    vmin = __reduce_min_sync(0xffffffffu, vmin);
    vmax = __reduce_max_sync(0xffffffffu, vmax);
    if (lane == 0) {
      s_box[warp][0] = umin;
      s_box[warp][1] = umax;
      s_box[warp][2] = vmin;
      s_box[warp][3] = vmax;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      umin = min(umin, s_box[w][0]);
      umax = max(umax, s_box[w][1]);
      vmin = min(vmin, s_box[w][2]);
      vmax = max(vmax, s_box[w][3]);
    }
    // raw frame: the box's left edge on a 4-float boundary of the frame
    // (a TMA requirement), in padded coordinates
    const bool raw = SINGLE && a.raw_frame;
    const int u0 = raw ? (((umin - PAD) & ~3) + PAD) : (umin & ~3);
    const int nbox = (vmax + D - vmin + ROI_BOX_H - 1) / ROI_BOX_H;
    const bool staged = (raw || a.tmaps != nullptr) && (umax + D - u0) <= ROI_W && nbox <= ROI_MAX_BOXES;

    if (staged) {
      if (threadIdx.x == 0 && !a.test_withhold_copy) {
        fence_proxy_async();  // earlier generic reads of s_roi before the async-proxy writes
        mbar_expect_tx(&s_bar, (uint32_t)(nbox * ROI_W * ROI_BOX_H * sizeof(float)));
        for (int b = 0; b < nbox; ++b) {
          if (raw)
            tma_load_2d(&s_roi[0][b * ROI_W * ROI_BOX_H], &a.zmap, u0 - PAD, vmin - PAD + b * ROI_BOX_H, &s_bar);
          else
            tma_load_2d(&s_roi[0][b * ROI_W * ROI_BOX_H], a.tmaps + ft, u0, vmin + b * ROI_BOX_H, &s_bar);
        }
      }
      const bool ok = mbar_wait(&s_bar, phase);
      if (__syncthreads_or(!ok)) {
        // the copy did not land within the bound: report and stop this CTA
        // after a second bounded wait, so no copy is left in flight
        if (threadIdx.x == 0) {
          set_error(a.ds, ERR_TIMEOUT, 4u, (uint32_t)tile, 0u);
          mbar_wait(&s_bar, phase);
        }
        return false;
      }
      phase ^= 1u;
      {
        // raw frame: y = z - b inside the frame, 0 outside (the copy filled
        // zeros there); then the shifted copy B[i] = A[i + 1]
        const int rows = nbox * ROI_BOX_H, x0 = u0 - PAD, y0 = vmin - PAD;
        const bool inside = !raw || (x0 >= 0 && y0 >= 0 && x0 + ROI_W <= P.W && y0 + rows <= P.H);
        float4* roi4 = reinterpret_cast<float4*>(&s_roi[0][0]);
        float* roiB = &s_roi[1][0];
        for (int e = threadIdx.x; e < rows * (ROI_W / 4); e += K1_THREADS) {
          float4 v = roi4[e];
          if (!raw) {
          } else if (inside) {
            v.x = __fsub_rn(v.x, P.bg);
            v.y = __fsub_rn(v.y, P.bg);
            v.z = __fsub_rn(v.z, P.bg);
            v.w = __fsub_rn(v.w, P.bg);
          } else {
            const int r = e / (ROI_W / 4), xc = x0 + (e - r * (ROI_W / 4)) * 4;
            const bool rin = (unsigned)(y0 + r) < (unsigned)P.H;
            v.x = rin && (unsigned)(xc + 0) < (unsigned)P.W ? __fsub_rn(v.x, P.bg) : 0.0f;
            v.y = rin && (unsigned)(xc + 1) < (unsigned)P.W ? __fsub_rn(v.y, P.bg) : 0.0f;
            v.z = rin && (unsigned)(xc + 2) < (unsigned)P.W ? __fsub_rn(v.z, P.bg) : 0.0f;
            v.w = rin && (unsigned)(xc + 3) < (unsigned)P.W ? __fsub_rn(v.w, P.bg) : 0.0f;
          }
          if (raw) roi4[e] = v;
          if (e > 0) roiB[4 * e - 1] = v.x;
          *reinterpret_cast<float2*>(roiB + 4 * e) = make_float2(v.y, v.z);
          roiB[4 * e + 2] = v.w;
        }
        __syncthreads();
      }
    }

    // Alg. 1 step U with the renormalised carried weight (Alg. 3 step 4)
    float lw[K1_PPT];
#pragma unroll
    for (int q = 0; q < K1_PPT; ++q) {
      const int jj = threadIdx.x + q * K1_THREADS;
      lw[q] = -INFINITY;
      if (jj < td.w) {
        float gxI[D];  // I gx(u), u = cx - R .. cx + R
        gauss_row_scaled<R>(floorf(s[q].x + 0.5f), s[q].x, P.c_psf, P.kappa, I[q], gxI);
        const float dy = floorf(s[q].y + 0.5f) - s[q].y;
        float ss;
        const bool frame_model = P.obs_model == 1;
        if (staged) {
          const int c = pu[q] - u0, o = (pv[q] - vmin) * ROI_W;
#ifdef PF_DEBUG
          // first and last floats the pairwise row loads touch
          if (o + c - (c & 1) < 0 || o + c - (c & 1) + 2 * R * ROI_W + 2 * R + 1 >= ROI_FLOATS + 4) {
            set_error(a.ds, ERR_DEBUG, 103u, (uint32_t)(o + c), (uint32_t)(ROI_FLOATS + 4));
            ss = 0.0f;
          } else
#endif
          {
            const float* base = (c & 1) ? &s_roi[1][o + c - 1] : &s_roi[0][o + c];
            ss = frame_model ? patch_ss_pairs<R, true>(base, gxI, dy, P.c_psf, P.kappa)
                             : patch_ss_pairs<R, false>(base, gxI, dy, P.c_psf, P.kappa);
          }
        } else if (raw) {
          ss = frame_model
                   ? patch_ss_raw<R, true>(a.zraw, P.W, P.H, P.bg, pu[q] - PAD, pv[q] - PAD, gxI, dy, P.c_psf, P.kappa)
                   : patch_ss_raw<R, false>(a.zraw, P.W, P.H, P.bg, pu[q] - PAD, pv[q] - PAD, gxI, dy, P.c_psf,
                                            P.kappa);
        } else {
#ifdef PF_DEBUG
          // the patch inside the padded frame (H + 2 PAD rows of P.pitch floats)
          if (pu[q] < 0 || pu[q] + 2 * R >= P.pitch || pv[q] < 0 || pv[q] + 2 * R >= P.H + 2 * PAD) {
            set_error(a.ds, ERR_DEBUG, 104u, (uint32_t)pu[q], (uint32_t)pv[q]);
            ss = 0.0f;
          } else
#endif
          {
            const float* base = a.ypad + ypad_off + (long long)pv[q] * P.pitch + pu[q];
            ss = frame_model ? patch_ss<R, true, false>(base, P.pitch, gxI, dy, P.c_psf, P.kappa)
                             : patch_ss<R, false, false>(base, P.pitch, gxI, dy, P.c_psf, P.kappa);
          }
        }
        const bool carried = VARIANTS && ((cmask >> (from_pred[q] ? 1 : 0)) & 1);
        lw[q] = fmaf(-ss, P.inv2so2, carried ? lw_t[g * Np + td.z + jj] : (from_pred[q] ? off_s : off_g));
        lw_t[g * Np + td.z + jj] = lw[q];
      }
    }

    // Per-tile partial sums for the group estimate, relative to the tile
    // max: each warp sums relative to its own max, and the 8 writers rescale
    // the warps' sums to the tile max (one barrier).
    int key = INT_MIN;
#pragma unroll
    for (int q = 0; q < K1_PPT; ++q)
      if (lw[q] == lw[q]) key = max(key, float_key(lw[q]));  // NaN does not count
    key = __reduce_max_sync(0xffffffffu, key);
    const float Mw = key == INT_MIN ? -INFINITY : key_float(key);
    float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < K1_PPT; ++q) {
      const float e = (lw[q] - Mw >= -87.0f) ? __expf(lw[q] - Mw) : 0.0f;
      v[0] += e;
      v[1] = fmaf(e, s[q].x, v[1]);
      v[2] = fmaf(e, s[q].y, v[2]);
      v[3] = fmaf(e, s[q].z, v[3]);
      v[4] = fmaf(e, s[q].w, v[4]);
      v[5] = fmaf(e, I[q], v[5]);
      v[6] = fmaf(e, e, v[6]);
    }
    int slot;
    const float x = warp_reduce8(v, lane, slot);
    if ((lane & 3) == 0) s_red[warp][slot] = x;
    if (lane == 0) s_key[warp] = key;
    __syncthreads();
    if (threadIdx.x < 8) {
      int kt = INT_MIN;
#pragma unroll
      for (int w = 0; w < NW; ++w) kt = max(kt, s_key[w]);
      const float Mt = key_float(kt);
      float r;
      if (threadIdx.x == 0) {
        r = Mt;
      } else {
        r = 0.0f;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const float mw = s_key[w] == INT_MIN ? -INFINITY : key_float(s_key[w]);
          float sc = (mw - Mt >= -87.0f) ? __expf(mw - Mt) : 0.0f;
          if (threadIdx.x == 7) sc *= sc;  // sums of e^2
          r = fmaf(sc, s_red[w][threadIdx.x - 1], r);
        }
      }
      a.tile_part[(long long)tile * 8 + threadIdx.x] = r;
    } else if (!FUSED && threadIdx.x == 8) {
      // raise the group maximum of the step (the resampler's quantisation scale)
      int kt = INT_MIN;
#pragma unroll
      for (int w = 0; w < NW; ++w) kt = max(kt, s_key[w]);
      if (kt != INT_MIN)  // (the group reloaded: no register held across the tile for it)
        atomicMax(&a.grp[P.group_off + __ldg(&a.tiles[tile].y)].mkey[k & 1], (uint32_t)kt ^ 0x80000000u);
    }
    // No barrier here: every shared buffer the next tile writes first (s_box,
    // then s_roi by TMA, s_red / s_key) is written only after that tile's
    // box barrier, which warp 0 reaches after its reads of s_red above.
    return true;
  };

  if constexpr (FUSED) {
    // Thread 0 schedules.  At the start of each task it claims, ahead of
    // need, the CTA's next tile and -- when the queue showed published work
    // and the CTA holds no position yet -- a queue position, so that both
    // round trips overlap the task.  At the next task boundary it runs the
    // held position's task if it is published, else the held tile; with no
    // tile left it waits (bounded) for its position, or claims one and
    // waits.  A held position depends only on earlier positions and on
    // tiles, which are always runnable, so every wait ends.
    __shared__ int s_code;
    const FusedSync fs{a.ring_stride};
    const int par = k & 1;
    const unsigned total = 2u * (unsigned)a.n_chunks;
    const bool worker = (int)blockIdx.x >= a.n_ring_blocks;
    const unsigned* q = a.rq + (size_t)par * 2 * a.n_chunks;
    unsigned* head = &a.sync[fs.rq_head(par)];
    int pend = -1;                  // held queue position (thread 0)
    unsigned ntile = 0u;            // held next tile (thread 0)
    bool have_tile = false;
    unsigned long long hint = 0ull; // (head, tail) as last read (thread 0)
    if (worker && threadIdx.x == 0) {
      ntile = atomicAdd(&a.sync[fs.tile_ctr(par)], 1u);
      have_tile = true;
    }
    for (;;) {
      if (threadIdx.x == 0) {
        int code = -1;
        if (worker) {
          if (pend >= 0) {
            const unsigned v = ld_acquire(q + pend);
            if (v != 0u) {
              code = (int)(v - 1u);
              pend = -1;
            }
          }
          if (code < 0 && have_tile && ntile < (unsigned)a.n_tiles) {
            code = (int)ntile;  // kind TASK_P = 0
            have_tile = false;
          }
          if (code < 0) {
            // no tile left: the held position, or a new one
            code = pend >= 0 ? rq_entry(a, par, (unsigned)pend) : rq_wait_claim(a, par);
            pend = -1;
          }
          // claims for the next boundary, in flight during this task
          if (code >= 0) {
            if (!have_tile && ntile < (unsigned)a.n_tiles) {
              ntile = atomicAdd(&a.sync[fs.tile_ctr(par)], 1u);
              have_tile = true;
            }
            const unsigned h = (unsigned)hint, t = (unsigned)(hint >> 32);
            if (pend < 0 && h < t && h < total && ntile < (unsigned)a.n_tiles) {
              const unsigned p = atomicAdd(head, 1u);
              pend = p < total ? (int)p : -1;
            }
            hint = *reinterpret_cast<volatile const unsigned long long*>(head);
          }
        }
        s_code = code;
      }
      __syncthreads();
      const int code = s_code;
      if (code < 0) break;
      const int kind = (int)((unsigned)code >> RQ_KIND_SHIFT), idx = code & ((1 << RQ_KIND_SHIFT) - 1);
      if (kind == TASK_P) {
        const int4 td = a.tiles[idx];
        if (threadIdx.x == 0) prefetch_tile(a, td, k, pv_prev, I_prev);
        if (!step_failed(a.ds)) {
          tile = idx;
          if constexpr (SINGLE)
            run_tile(a.p0, td);
          else
            run_tile(a.trk[td.x], td);
        }
        __syncthreads();  // the tile's log-weights and partial sums are written
        const int gi = (SINGLE ? a.p0.group_off : a.trk[td.x].group_off) + td.y;
        if (threadIdx.x == 0) {
          __threadfence();
          const unsigned prev = atomicAdd(&a.sync[fs.pdone(par, gi)], 1u);
          s_code = (prev + 1u == (unsigned)a.gd[gi].tile_count) ? 1 : 0;
        }
        __syncthreads();
        if (s_code) fused_group_tiles_done(a, k, gi);
      } else if (kind == TASK_A) {
        fused_task_a(a, k, idx, s_dyn);
      } else {
        fused_task_b(a, k, idx, s_dyn);
      }
      __syncthreads();  // the next task reuses the shared buffers and s_code
    }
    // the last CTA to leave advances the step index of every track
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&a.sync[fs.exit_ctr(par)], 1u);
      s_last = (prev + 1u == gridDim.x) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      for (int t = threadIdx.x; t < a.n_tracks; t += K1_THREADS) a.ts[t].k = k + 1;
    }
    return;
  }

  // first tile by block index, the rest from a counter (reset by the
  // resampler), so CTAs finish together however many tiles each ran
  if constexpr (!FUSED) {  // (the one-launch step has returned above)
    for (int it = 0; tile < a.n_tiles; ++it) {
      const int4 td = a.tiles[tile];
      if (threadIdx.x == 0) {
        const int nt = stride + atomicAdd(a.tile_ctr, 1);
        s_next[it & 1] = nt;
        if (nt < a.n_tiles) prefetch_tile(a, a.tiles[nt], k, pv_prev, I_prev);
      }
      bool ok;
      if constexpr (SINGLE)
        ok = run_tile(a.p0, td);
      else
        ok = run_tile(a.trk[td.x], td);
      if (!ok) return;
      tile = s_next[it & 1];  // written before run_tile's barriers; rewritten two tiles later
    }
  }
}

// ==================================================================== resample
// #{j in [0, Np) : T_j < S}, the number of outputs that go to items whose
// boundary is below S (0 <= S <= Q).  T_j < S exactly when j < x =
// (S Np - F) / Q, so the count is ceil(x) clamped to [0, Np].  The FP32
// estimate fma(S, Np / Q, -u 2^-32) is within Np 2^-21 < 1/2 of x (S and Q
// each converted within 2^-23, the quotient and the product rounded, u
// truncated to 24 bits, Np <= 2^20), so its ceiling is the count or one
// off, and one comparison each way (Thresholds::le, whose result is that
// of the exact form) settles it, without branches.  Both corrections at
// once would break that bound: reported.
__device__ __forceinline__ int count_below(const Thresholds& th, unsigned long long S, float inv_Q, int Np,
                                           uint32_t u, DevState* ds) {
  const float Sf = u64_to_float_approx(S);
  const float Npf = (float)Np;
  const float est = fminf(fmaxf(fmaf(Sf, Npf * inv_Q, -(float)(u >> 8) * 5.9604645e-8f), 0.0f), Npf);
  const float c0 = __fadd_ru(est, 8388608.0f) - 8388608.0f;  // ceil: est is in [0, 2^20]
  const bool up = c0 < Npf && !th.le(S, Sf, c0);              // T_c0 < S
  const bool dn = c0 > 0.0f && th.le(S, Sf, c0 - 1.0f);       // T_(c0-1) >= S
  if (up && dn) set_error(ds, ERR_INVARIANT, 3u, (uint32_t)S, (uint32_t)c0);
  const float c = c0 + (up ? 1.0f : 0.0f) - (dn ? 1.0f : 0.0f);
  return S == 0 ? 0 : __float_as_int(c + 8388608.0f) - 0x4B000000;
}

// Shared-memory accesses through 32-bit shared-window addresses (the merge
// helpers are not inlined, and a generic pointer would make every access a
// generic one).
__device__ __forceinline__ unsigned long long lds_u64(uint32_t addr) {
  unsigned long long v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// A store to the shared memory of CTA `rank` of the cluster, at the
// address `addr` has in this CTA's window.
__device__ __forceinline__ void sts_cluster_u32(uint32_t addr, uint32_t rank, uint32_t v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(addr), "r"(rank));
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(remote), "r"(v) : "memory");
}
// The two halves of a cluster barrier: stores before the arrival are
// visible to every CTA of the cluster after its wait.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
// X_i = s_incl[pad8(i)] at shared address base
__device__ __forceinline__ unsigned long long incl_at(uint32_t base, int i) {
  return lds_u64(base + 8u * (uint32_t)pad8(i));
}

// Block-wide split of a merge at diagonal p: the number of items among its
// first p positions, for items i < n with boundaries X_i = s_incl[pad8(i)]
// and outputs j0 + b, b < no, with thresholds T: the largest i in
// [max(0, p - no), min(p, n)] with X_{i-1} <= T_{j0+p-i}.  A
// NTR-ary search that every thread of the block (NTR threads) enters.
template <int NTR>
__device__ __noinline__ int merge_split(uint32_t s_incl, const Thresholds& th, int j0, int n, int no, int p) {
  int lo = max(0, p - no), hi = min(p, n);
  while (lo < hi) {
    const int m = hi - lo;
    const bool fine = m <= NTR;  // then candidates lo + 1 .. hi, else NTR evenly spaced
    const int c = fine ? lo + 1 + (int)threadIdx.x : lo + (int)(((long long)(threadIdx.x + 1) * m) / NTR);
    const bool ok = (!fine || (int)threadIdx.x < m) && th.le(incl_at(s_incl, c - 1), (uint32_t)(j0 + p - c));
    const int cnt = __syncthreads_count(ok);  // the predicate holds for a prefix of the candidates
    if (fine) {
      lo += cnt;
      hi = lo;
    } else {
      const int nlo = cnt == 0 ? lo : lo + (int)(((long long)cnt * m) / NTR);
      const int nhi = cnt == NTR ? hi : lo + (int)(((long long)(cnt + 1) * m) / NTR) - 1;
      lo = nlo;
      hi = nhi;
    }
  }
  return lo;
}

// The merge of one resampler sub-chunk: n items with boundaries
// X_i = s_incl[pad8(i)] against outputs j in [jlo, jhi); ancestors
// obase_sub + item, stored to anc[j].  Every thread of the block enters.
// (Not inlined: it runs with registers of its own.)
template <int NTR>
__device__ __noinline__ void merge_windows(const unsigned long long* __restrict__ s_incl_p, uint32_t* __restrict__ s_out_p,
                                           const Thresholds& th_s, int jlo, int jhi, int n,
                                           unsigned long long obase_sub, uint32_t* __restrict__ anc) {
  constexpr int WIN = 2 * NTR * RS_ITEMS;
  const Thresholds th = th_s;
  const uint32_t s_incl = (uint32_t)__cvta_generic_to_shared(s_incl_p);
  const uint32_t s_out = (uint32_t)__cvta_generic_to_shared(s_out_p);
  // Merge path over the item boundaries X_i = S_{i+1} (s_incl) and the
  // thresholds Y_j = T_j of this sub-chunk's outputs j in [jlo, jhi):
  // output j takes the first item i with T_j < S_{i+1}.  The merged
  // sequence (n items, no outputs) is cut into windows of at most WIN
  // positions, each split at its diagonal by a block-wide search, so that
  // every item and output is merged once however the weight is spread
  // over the CTAs; within a window each thread merges an equal slice.  A
  // window's ancestors are staged in shared memory and stored with
  // consecutive threads writing consecutive outputs.
  const int no = jhi - jlo, Lt = n + no;
  int ia0 = 0, ib0 = 0;  // items and outputs merged before the window
  for (int p0 = 0; p0 < Lt; p0 += WIN) {
    const int p1 = min(Lt, p0 + WIN);
    const int ia1 = p1 == Lt ? n : merge_split<NTR>(s_incl, th, jlo, n, no, p1);
    const int nw = ia1 - ia0, mw = (p1 - ia1) - ib0, L = p1 - p0;
    const int jw = jlo + ib0;
    const int d0 = (int)(((long long)L * threadIdx.x) / NTR);
    const int d1 = (int)(((long long)L * (threadIdx.x + 1)) / NTR);
    // largest ia in [max(0, d0 - mw), min(d0, nw)] whose items all precede
    // output d0 - ia of the window in the merge (X_{ia0+ia-1} <= Y_{jw+d0-ia})
    int lo2 = max(0, d0 - mw), hi2 = min(d0, nw);
    while (lo2 < hi2) {
      const int mid = (lo2 + hi2 + 1) >> 1;  // candidate number of items consumed
      if (th.le(incl_at(s_incl, ia0 + mid - 1), (uint32_t)(jw + d0 - mid))) lo2 = mid;
      else hi2 = mid - 1;
    }
    int ia = lo2, ib = d0 - lo2;
    if (ib < mw) {
      // T and its remainder at output jw + ib, then advance incrementally;
      // the current item's boundary stays in a register (past the window's
      // last item it counts as unbounded)
      uint32_t jj = (uint32_t)(jw + ib);
      unsigned long long num = (unsigned long long)jj * th.B + th.F0;
      unsigned long long qd = th.Np > 1 ? __umul64hi(num, th.M) : num;
      uint32_t rem = (uint32_t)(num - qd * th.Np);
      unsigned long long Tj = (unsigned long long)jj * th.A + th.F1 + qd;
      unsigned long long X = ia < nw ? incl_at(s_incl, ia0 + ia) : ~0ull;
      for (int dd = d0; dd < d1; ++dd) {
        if (ib < mw && Tj < X) {
          sts_u32(s_out + 4u * (uint32_t)pad8(ib), (uint32_t)(obase_sub + ia0 + ia));
          ++ib;
          rem += th.B;
          Tj += th.A;
          if (rem >= th.Np) {
            rem -= th.Np;
            Tj += 1;
          }
        } else {
          ++ia;
          X = ia < nw ? incl_at(s_incl, ia0 + ia) : ~0ull;
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < mw; e += NTR) anc[jw + e] = lds_u32(s_out + 4u * (uint32_t)pad8(e));
    __syncthreads();
    ia0 = ia1;
    ib0 += mw;
  }
}

// ================================================================ fused step
// One persistent launch per step.  Its CTAs take propagate + weight tiles
// (P) from a counter, and resampling tasks from a ready queue as soon as
// they can run: the tile that completes a group publishes the group maximum
// and queues the group's chunk tasks A (quantise RS_CHUNK slots, sum their
// weight codes); the A task that completes a group publishes the group
// total, queues its chunk tasks B (scan and merge, Alg. 3 step 7), and
// finishes the group's statistics (step 6); the track's last group runs
// the global step (steps 8-10, and 1-2 of the next step).  A CTA takes a
// ready task before a new tile, so no task ever waits for another; the only
// wait is that of a CTA with no tiles left for the next ready task, and
// every wait is bounded (0.2 s of %globaltimer: ERR_TIMEOUT, and the tasks
// after it skip their work).  Counters and queue entries are per step
// parity and cleared by the leading blocks of the step before.

// An earlier kernel or task gave up (bounded wait) or met an out-of-range
// ancestor: the weights mean nothing, later tasks skip their work.
__device__ __forceinline__ bool step_failed(const DevState* ds) {
  return (*reinterpret_cast<volatile const unsigned int*>(&ds->err) & (ERR_TIMEOUT | ERR_INDEX)) != 0u;
}

// Thread 0: the task published at queue position pos (waiting, bounded,
// for its entry: the position was claimed after it was counted, or ahead of
// it once no tiles were left), or -1.
__device__ __noinline__ int rq_entry(const K1Args& a, int par, unsigned pos) {
  const unsigned* q = a.rq + (size_t)par * 2 * a.n_chunks + pos;
  unsigned v = ld_acquire(q);
  if (v == 0u) {
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    while ((v = ld_acquire(q)) == 0u) {
      if (step_failed(a.ds)) return -1;
      if (global_ns() - t0 > 200000000ull) {
        set_error(a.ds, ERR_TIMEOUT, 9u, pos, 0u);
        return -1;
      }
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
    }
  }
  return (int)(v - 1u);
}

// Thread 0, while tiles are left: one attempt at the next published ready
// task; -1 if none is published or another CTA took it first.
__device__ __noinline__ int rq_try_claim(const K1Args& a, int par) {
  const FusedSync fs{a.ring_stride};
  unsigned* head = &a.sync[fs.rq_head(par)];
  const unsigned long long ht = *reinterpret_cast<volatile const unsigned long long*>(head);  // (head, tail)
  const unsigned h = (unsigned)ht, t = (unsigned)(ht >> 32);
  if (h >= t || atomicCAS(head, h, h + 1u) != h) return -1;
  return rq_entry(a, par, h);
}

// Thread 0, once no tiles are left: the next queue position, whether its
// task is published yet or not; -1 once every resampling task is taken (the
// CTA then leaves).
__device__ __noinline__ int rq_wait_claim(const K1Args& a, int par) {
  const FusedSync fs{a.ring_stride};
  const unsigned total = 2u * (unsigned)a.n_chunks;
  if (*reinterpret_cast<volatile const unsigned*>(&a.sync[fs.rq_head(par)]) >= total) return -1;
  const unsigned pos = atomicAdd(&a.sync[fs.rq_head(par)], 1u);
  if (pos >= total) return -1;
  return rq_entry(a, par, pos);
}

// Publish the chunk tasks of group d (kind TASK_A or TASK_B): the whole CTA
// enters; the caller has written what the tasks read and fenced.
__device__ __forceinline__ void rq_push_group(const K1Args& a, int par, const GroupDesc& d, int kind, int* s_pos) {
  const FusedSync fs{a.ring_stride};
  if (threadIdx.x == 0) *s_pos = (int)atomicAdd(&a.sync[fs.rq_tail(par)], (unsigned)d.chunk_count);
  __syncthreads();
  unsigned* q = a.rq + (size_t)par * 2 * a.n_chunks;
  for (int c = threadIdx.x; c < d.chunk_count; c += K1_THREADS) {
    __threadfence();
    q[*s_pos + c] = (((unsigned)kind << RQ_KIND_SHIFT) | (unsigned)(d.chunk_begin + c)) + 1u;
  }
}

// Thread 0: wait (bounded) until the leading blocks of this launch are done.
__device__ __noinline__ int fused_wait_ring(const K1Args& a, int par, int gi) {
  const FusedSync fs{a.ring_stride};
  const unsigned* p = &a.sync[fs.ring_done(par)];
  const unsigned target = (unsigned)a.n_ring_blocks;
  if (ld_acquire(p) >= target) return 1;
  const unsigned long long t0 = global_ns();
  while (ld_acquire(p) < target) {
    __nanosleep(128);
    if (global_ns() - t0 > 200000000ull) {
      set_error(a.ds, ERR_TIMEOUT, 7u, (uint32_t)gi, ld_acquire(p));
      return 0;
    }
  }
  return 1;
}

// The chunk's log-weights (items lo + threadIdx.x * RS_ITEMS .. + RS_ITEMS
// of the group, -inf past its end), through L2: other CTAs of this launch
// wrote them.
__device__ __forceinline__ void fused_load_items(const float* __restrict__ lw, long long base, int i0, int hi,
                                                 float (&v)[RS_ITEMS]) {
  if (((base + i0) & 3) == 0 && i0 + RS_ITEMS <= hi) {
    const float4 x0 = __ldcg(reinterpret_cast<const float4*>(lw + base + i0));
    const float4 x1 = __ldcg(reinterpret_cast<const float4*>(lw + base + i0 + 4));
    v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
    v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
  } else {
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) v[r] = (i0 + r < hi) ? __ldcg(lw + base + i0 + r) : -INFINITY;
  }
}

// The tile that completes group gi: the group maximum of its log-weights
// from the tiles' maxima (NaN ignored), then the group's A tasks.
__device__ __noinline__ void fused_group_tiles_done(const K1Args& a, int k, int gi) {
  __shared__ float s_f[K1_THREADS / 32];
  __shared__ int s_pos;
  const GroupDesc d = a.gd[gi];
  float m = -INFINITY;
  for (int t = threadIdx.x; t < d.tile_count; t += K1_THREADS)
    m = fmaxf(m, __ldcg(&a.tile_part[(long long)(d.tile_begin + t) * 8]));
  const float M = block_max<K1_THREADS>(m, s_f);
  if (threadIdx.x == 0) {
    a.grp[gi].M = M;
    __threadfence();
  }
  rq_push_group(a, k & 1, d, TASK_A, &s_pos);
}

// The A task that completes group gi: the group total of the weight codes
// and Alg. 1's decision, the group's B tasks, then the group estimate and
// ESS from the tile partial sums (Alg. 3 step 6) and the track's ticket;
// the track's last group runs the global step.
__device__ __noinline__ void fused_group_finalize(const K1Args& a, int k, int gi, float M, unsigned char* smem) {
  __shared__ int s_flag, s_pos;
  __shared__ unsigned long long s_w[K1_THREADS / 32];
  __shared__ float s_stat[K1_THREADS / 32][8];
  const int par = k & 1;
  const GroupDesc d = a.gd[gi];
  const TrackParams& P = a.trk[d.track];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool ess = P.resample_rule == 1;
  unsigned long long q = 0, e1 = 0, e2 = 0;
  for (int c = threadIdx.x; c < d.chunk_count; c += K1_THREADS) {
    const long long cc = d.chunk_begin + c;
    q += __ldcg(&a.chunk_q[4 * cc]);
    if (ess) {
      e1 += __ldcg(&a.chunk_q[4 * cc + 1]);
      e2 += __ldcg(&a.chunk_q[4 * cc + 2]);
    }
  }
  const unsigned long long Q = block_sum_u64<K1_THREADS>(q, s_w);
  const unsigned long long E1 = ess ? block_sum_u64<K1_THREADS>(e1, s_w) : 0ull;
  const unsigned long long E2 = ess ? block_sum_u64<K1_THREADS>(e2, s_w) : 0ull;
  const bool resample = !ess || Q == 0 || ess_below(E1, E2, (uint32_t)P.Np, P.ess_t);
  GroupState& G = a.grp[gi];
  if (warp == 0) {
    // each chunk's offset on the group's prefix-sum axis (exclusive sums of
    // the chunk totals, in chunk order)
    unsigned long long carry = 0;
    for (int c0 = 0; c0 < d.chunk_count; c0 += 32) {
      const int c = c0 + lane;
      const unsigned long long x = c < d.chunk_count ? __ldcg(&a.chunk_q[4 * (long long)(d.chunk_begin + c)]) : 0ull;
      unsigned long long y = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += t;
      }
      if (c < d.chunk_count) a.chunk_q[4 * (long long)(d.chunk_begin + c) + 3] = carry + y - x;
      carry += __shfl_sync(0xffffffffu, y, 31);
    }
    if (lane == 0) {
      G.Q = Q;
      G.carry_next = resample ? 0 : 1;
      if (Q != 0) {
        // the thresholds of the group's outputs (its resampling uniform word:
        // Philox stream RESAMPLE, group, step)
        const uint32_t u =
            philox(P.key0, P.key1, make_uint4((uint32_t)d.g, 0u, (uint32_t)k, P.tag | (ST_RESAMPLE << 4))).x;
        Thresholds th;
        th.init_magic(Q, (uint32_t)P.Np, u, P.m_Np);
        G.u = u;
        G.th_A = th.A;
        G.th_F1 = th.F1;
        G.th_M = th.M;
        G.th_B = th.B;
        G.th_F0 = th.F0;
        G.th_Np = th.Np;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) __threadfence();
  rq_push_group(a, par, d, TASK_B, &s_pos);
  // the leading blocks read the previous step's group estimates: they finish first
  if (threadIdx.x == 0) s_flag = fused_wait_ring(a, par, gi);
  float acc[7] = {0, 0, 0, 0, 0, 0, 0};
  if (Q != 0) {
    for (int t = threadIdx.x; t < d.tile_count; t += K1_THREADS) {
      const float* tp = a.tile_part + (long long)(d.tile_begin + t) * 8;
      const float Mt = __ldcg(tp);
      if (!(Mt - M >= -87.0f)) continue;
      const float sc = __expf(Mt - M);
#pragma unroll
      for (int j = 0; j < 6; ++j) acc[j] = fmaf(sc, __ldcg(tp + 1 + j), acc[j]);
      acc[6] = fmaf(sc * sc, __ldcg(tp + 7), acc[6]);
    }
  }
#pragma unroll
  for (int j = 0; j < 7; ++j) acc[j] = warp_sum(acc[j]);
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < 7; ++j) s_stat[warp][j] = acc[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    float t7[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int w = 0; w < K1_THREADS / 32; ++w)
      for (int j = 0; j < 7; ++j) t7[j] += s_stat[w][j];
    const bool okw = (Q != 0) && t7[0] > 0.0f;
    for (int j = 0; j < 5; ++j) G.xs[j] = okw ? t7[1 + j] / t7[0] : 0.0f;
    G.ess = okw ? t7[0] * t7[0] / t7[6] : 0.0f;
    __threadfence();
    const unsigned prev = atomicAdd(&a.ts[d.track].ticket, 1u);
    s_flag = (prev + 1u == (unsigned)P.G) ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  if (s_flag) {
    const GlobalArgs ga{a.trk, a.ts, a.grp, a.ring, a.ring_next, a.ring_stride, a.exo_next, a.hist, a.ghist,
                        a.history, 1, a.ds, 1};
    global_step<K1_THREADS>(ga, d.track, *reinterpret_cast<GlobalScratch*>(smem));
    if (threadIdx.x == 0) a.ts[d.track].ticket = 0u;
  }
}

// Task A of chunk ci: quantise the chunk's log-weights against the group
// maximum (Alg. 3 step 7's fixed-point weights) and publish their sum; the
// group's last chunk finalises the group.
__device__ __noinline__ void fused_task_a(const K1Args& a, int k, int ci, unsigned char* smem) {
  __shared__ int s_last;
  __shared__ unsigned long long s_w[K1_THREADS / 32];
  const FusedSync fs{a.ring_stride};
  const int par = k & 1;
  const int4 ch = a.chunks[ci];  // (track, group, first slot, items)
  const GroupDesc d = a.gd[ch.y];
  const TrackParams& P = a.trk[ch.x];
  const bool ok = !step_failed(a.ds);
  const bool ess = P.resample_rule == 1;
  const float M = __ldcg(&a.grp[ch.y].M);
  unsigned long long qs = 0, e1 = 0, e2 = 0;
  if (ok) {
    const float* __restrict__ lw = (k & 1) ? a.lw1 : a.lw;
    float v[RS_ITEMS];
    fused_load_items(lw, d.base, ch.z + (int)threadIdx.x * RS_ITEMS, ch.z + ch.w, v);
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
      const unsigned long long q = quantize(v[r], M, a.qc);
      qs += q;
      if (ess) {
        const unsigned long long c = q >> 20;
        e1 += c;
        e2 += c * c;
      }
    }
  }
  qs = block_sum_u64<K1_THREADS>(qs, s_w);
  if (ess) {
    e1 = block_sum_u64<K1_THREADS>(e1, s_w);
    e2 = block_sum_u64<K1_THREADS>(e2, s_w);
  }
  if (threadIdx.x == 0) {
    a.chunk_q[4 * (long long)ci] = qs;
    a.chunk_q[4 * (long long)ci + 1] = e1;
    a.chunk_q[4 * (long long)ci + 2] = e2;
    __threadfence();
    const unsigned prev = atomicAdd(&a.sync[fs.adone(par, ch.y)], 1u);
    s_last = (ok && prev + 1u == (unsigned)d.chunk_count) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) fused_group_finalize(a, k, ch.y, M, smem);
}

// Task B of chunk ci: the exact systematic resampling (Alg. 3 step 7) of the
// outputs whose thresholds fall in this chunk: a block-wide scan of the
// chunk's codes from the sum of the chunks before it, then the merge path
// of the two-launch resampler.
__device__ __noinline__ void fused_task_b(const K1Args& a, int k, int ci, unsigned char* smem) {
  __shared__ int s_jlo, s_jhi;
  __shared__ unsigned long long s_w[K1_THREADS / 32], s_sb;
  __shared__ uint32_t s_u;
  __shared__ Thresholds s_th;
  const int4 ch = a.chunks[ci];
  const GroupDesc d = a.gd[ch.y];
  const TrackParams& P = a.trk[ch.x];
  const int Np = d.Np, lo = ch.z, n = ch.w;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (step_failed(a.ds)) return;
  const unsigned long long Q = __ldcg(&a.grp[ch.y].Q);
  const bool keep = __ldcg(&a.grp[ch.y].carry_next) != 0;
  const unsigned long long obase = (unsigned long long)d.g * (unsigned long long)Np;
  uint32_t* __restrict__ anc = a.anc + (k & 1) * a.anc_stride + d.base;
  if (Q == 0 || keep) {
    // no finite weight, or Alg. 1's test keeps the particles: identity
    for (int i = lo + threadIdx.x; i < lo + n; i += K1_THREADS) anc[i] = (uint32_t)(obase + i);
    return;
  }
  const float M = __ldcg(&a.grp[ch.y].M);
  if (threadIdx.x == 0) {
    // the group's thresholds and this chunk's offset, from its finalisation
    const GroupState& G = a.grp[ch.y];
    s_sb = __ldcg(&a.chunk_q[4 * (long long)ci + 3]);
    s_u = __ldcg(&G.u);
    s_th.A = __ldcg(&G.th_A);
    s_th.F1 = __ldcg(&G.th_F1);
    s_th.M = __ldcg(&G.th_M);
    s_th.B = __ldcg(&G.th_B);
    s_th.F0 = __ldcg(&G.th_F0);
    s_th.Np = __ldcg(&G.th_Np);
    s_th.init_filter();
  }
  (void)P;
  unsigned long long* s_incl = reinterpret_cast<unsigned long long*>(smem);
  uint32_t* s_out = reinterpret_cast<uint32_t*>(smem + sizeof(unsigned long long) * pad8(RS_CHUNK));
  const float* __restrict__ lw = (k & 1) ? a.lw1 : a.lw;
  const int i0 = (int)threadIdx.x * RS_ITEMS;
  float v[RS_ITEMS];
  fused_load_items(lw, d.base, lo + i0, lo + n, v);
  unsigned long long qv[RS_ITEMS];
  unsigned long long tsum = 0;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    qv[r] = quantize(v[r], M, a.qc);
    tsum += qv[r];
  }
  // exclusive scan of the thread totals: warp shuffles, then warps
  unsigned long long x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  unsigned long long wpre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < K1_THREADS / 32; ++w) {
    const unsigned long long y = s_w[w];
    if (w < warp) wpre += y;
    tot += y;
  }
  const unsigned long long Sb = s_sb;
  {
    unsigned long long S = Sb + wpre + (x - tsum);
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
      S += qv[r];
      s_incl[pad8(i0 + r)] = S;
    }
  }
  if (threadIdx.x == 0) {
    const Thresholds th = s_th;
    const float inv_Q = 1.0f / u64_to_float_approx(Q);
    s_jlo = count_below(th, Sb, inv_Q, Np, s_u, a.ds);
    s_jhi = count_below(th, Sb + tot, inv_Q, Np, s_u, a.ds);
  }
  __syncthreads();
  merge_windows<K1_THREADS>(s_incl, s_out, s_th, s_jlo, s_jhi, n, obase + lo, anc);
}

// Wait (bounded, 0.2 s) until the G groups of a track have taken their
// tickets; 0 after a failed propagate launch (the groups skip their work and
// their tickets) or a timeout.
__device__ __forceinline__ int wait_tickets(const unsigned* tk, unsigned G, DevState* ds) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(tk) : "memory");
  const unsigned long long t0 = global_ns();
  while (v < G) {
    if ((*reinterpret_cast<volatile const unsigned int*>(&ds->err) & (ERR_TIMEOUT | ERR_INDEX)) != 0u) return 0;
    __nanosleep(64);
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(tk) : "memory");
    if (global_ns() - t0 > 200000000ull) {
      set_error(ds, ERR_TIMEOUT, 11u, v, G);
      return 0;
    }
  }
  return 1;
}

// The global step of a one-track resampling launch, by one CTA, once the
// track's G groups have taken their tickets (a failed propagate launch or a
// timeout ends the wait without a global step).  What the groups do not
// write is read before the wait.
template <int NT>
__device__ __forceinline__ void global_step_when_reported(const GlobalArgs& g, DevState* ds, GlobalScratch& sc) {
  __shared__ int s_ok;
  GlobalIn<NT> in;
  global_load<NT>(g, 0, in);
  if (threadIdx.x == 0) s_ok = wait_tickets(&g.ts[0].ticket, (unsigned)in.G, ds);
  __syncthreads();
  if (s_ok) {
    global_step_core<NT>(g, 0, sc, in);
    if (threadIdx.x == 0) g.ts[0].ticket = 0u;
  }
}

// The lean resampler's mark array follows the global step's scratch in
// dynamic shared memory (rank 0 may run the global step while the other
// CTAs of its cluster mark its output positions).
constexpr size_t RS_MARK_OFF = (sizeof(GlobalScratch) + 15) / 16 * 16;

// Resampler: one thread-block cluster per group, each CTA a contiguous chunk
// of the group's slots (a multiple of 8), processed in sub-chunks of SUB
// items; thread t owns the RS_ITEMS consecutive items [t*RS_ITEMS, ...).

// LEAN: every CTA's chunk fits in its registers (one sub-chunk), no group
// resamples by Alg. 1's test and no weight codes are stored (the common
// filter step, and pf_resample without codes) -- with the other paths
// compiled out (a smaller kernel: the resampler is latency-bound, and
// instruction fetch leads its stalls).
template <int NTR, bool LEAN>
__global__ void __launch_bounds__(NTR, NTR >= 512 ? 2 : 8) k_resample(const __grid_constant__ ResampleArgs a) {
  constexpr int SUB = NTR * RS_ITEMS;  // items per sub-chunk
  constexpr int SUB_PAD = pad8(SUB);
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int grp = blockIdx.x / C;
  if (a.fuse_global == 2 && grp >= a.n_groups) {
    // the extra cluster of a one-track step: its first CTA runs the
    // track's global step once every group has reported; nothing waits on
    // it within the launch
    extern __shared__ unsigned long long s_dyn_gs[];
    grid_dep_wait();
    if (rank == 0) global_step_when_reported<NTR>(a.glob, a.ds, *reinterpret_cast<GlobalScratch*>(s_dyn_gs));
    grid_dep_launch();
    return;
  }
  const GroupDesc d = a.gd[grp];
  const int Np = d.Np;
  const int chunk = ((Np + C - 1) / C + 7) & ~7;
  const int lo = min(rank * chunk, Np), hi = min(lo + chunk, Np);
  const bool single = LEAN || (hi - lo) <= SUB;  // the whole chunk stays in registers
  // In a filter step: the track's step index (read before the cluster
  // barrier that precedes every ticket below, since the track's global step,
  // run by the last ticket holder, advances it), which picks the log-weight
  // buffer and the resampling uniform.
  const TrackParams* __restrict__ Pt = a.glob.trk ? a.glob.trk + d.track : nullptr;
  const int kk = a.u_arr ? 0 : a.glob.ts[d.track].k;
  const float* __restrict__ lw = ((a.lw1 && (kk & 1)) ? a.lw1 : a.lw) + d.base;
  const bool ess_rule = !LEAN && Pt && Pt->resample_rule == 1;
  const bool vec = ((d.base & 3) == 0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  __shared__ float s_pub_max;
  __shared__ unsigned long long s_pub_q;
  __shared__ unsigned long long s_pub_e[2];
  __shared__ float s_f[NTR / 32];
  __shared__ unsigned long long s_w[NTR / 32];
  __shared__ float s_stat[NTR / 32][8];
  __shared__ int s_jlo, s_jhi;
  __shared__ Thresholds s_th;
  // dynamic: inclusive prefixes of a sub-chunk's items, then a window of
  // ancestors staged for coalesced stores.  Both are indexed through pad8
  // (one spare element per 8): a thread's 8 consecutive items then start 9
  // elements after its neighbour's, spreading a warp over the banks.
  extern __shared__ __align__(16) unsigned long long s_dyn_rs[];
  unsigned long long* s_incl = s_dyn_rs;
  uint32_t* s_out = reinterpret_cast<uint32_t*>(s_dyn_rs + SUB_PAD);
  // LEAN: one entry per output position of this CTA (NTR RS_ITEMS), 0 or
  // the 1-based item whose outputs start there
  uint32_t* s_mark = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(s_dyn_rs) + RS_MARK_OFF);

  float v[RS_ITEMS];
  auto load_sub = [&](int sub) {
    const int i0 = sub + (int)threadIdx.x * RS_ITEMS;
    if (vec && i0 + RS_ITEMS <= hi) {
      const float4 x0 = *reinterpret_cast<const float4*>(lw + i0);
      const float4 x1 = *reinterpret_cast<const float4*>(lw + i0 + 4);
      v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
      v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
    } else {
#pragma unroll
      for (int r = 0; r < RS_ITEMS; ++r) v[r] = (i0 + r < hi) ? lw[i0 + r] : -INFINITY;
    }
  };

  // The group's resampling uniform word (Philox stream RESAMPLE, group,
  // step).  In a filter step it depends only on the seed and the step index
  // (set by the previous step's global step, complete before the propagate
  // kernel ran), so it is drawn before waiting for the propagate kernel.
  if constexpr (LEAN) {
    uint4* m4 = reinterpret_cast<uint4*>(s_mark) + 2 * threadIdx.x;
    m4[0] = make_uint4(0u, 0u, 0u, 0u);  // before the cluster barrier that precedes any marking
    m4[1] = make_uint4(0u, 0u, 0u, 0u);
  }
  uint32_t u = 0;
  if (!a.u_arr)
    u = philox(Pt->key0, Pt->key1, make_uint4((uint32_t)d.g, 0u, (uint32_t)kk, Pt->tag | (ST_RESAMPLE << 4))).x;
  grid_dep_wait();
  if (a.u_arr) u = a.u_arr[grp];
  if (a.tile_ctr && blockIdx.x == 0 && threadIdx.x == 0) *a.tile_ctr = 0;  // for the next propagate launch
  // A propagate launch that timed out or met an out-of-range ancestor left
  // weights that mean nothing: resample nothing.  Only the kernels before
  // this one set these two bits, so every CTA of a cluster decides alike.
  if (a.ds && (*reinterpret_cast<volatile const unsigned int*>(&a.ds->err) & (ERR_TIMEOUT | ERR_INDEX)) != 0u) return;

  // group maximum: from the propagate tiles' maxima in a filter step, else
  // over the cluster (the same set of log-weights either way, NaN ignored)
  float M = -INFINITY;
  if (single) load_sub(lo);  // the CTA's items, for the quantisation below
  if (a.tile_part != nullptr) {
    // the largest tile maximum, raised by the propagate tiles (NaN and
    // tiles with no finite weight never raise it)
    const uint32_t mk = __ldcg(&a.gs[grp].mkey[kk & 1]);
    M = mk == 0u ? -INFINITY : key_float((int)(mk ^ 0x80000000u));
    if (rank == 0 && threadIdx.x == 0) a.gs[grp].mkey[(kk + 1) & 1] = 0u;  // for the next step's tiles
  } else {
    float m = -INFINITY;
    for (int sub = lo; sub < hi; sub += SUB) {
      if (!single) load_sub(sub);
#pragma unroll
      for (int r = 0; r < RS_ITEMS; ++r) m = fmaxf(m, v[r]);
    }
    m = block_max<NTR>(m, s_f);
    if (threadIdx.x == 0) s_pub_max = m;
    cl.sync();
    for (int r = 0; r < C; ++r) M = fmaxf(M, *cl.map_shared_rank(&s_pub_max, r));
  }

  // this CTA's total weight code, then the cluster prefix and group total;
  // under Alg. 1's test also the sums of c = q >> 20 and c^2
  unsigned long long qs = 0, e1 = 0, e2 = 0;
  unsigned long long qv[RS_ITEMS] = {0, 0, 0, 0, 0, 0, 0, 0};  // 0 on a CTA past the group's end
  for (int sub = lo; sub < hi; sub += SUB) {
    if (!single) load_sub(sub);
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
      qv[r] = quantize(v[r], M, a.qc);
      qs += qv[r];
      if (ess_rule) {
        const unsigned long long c = qv[r] >> 20;
        e1 += c;
        e2 += c * c;
      }
    }
  }
  // LEAN: one scan of the thread totals gives both the CTA total and each
  // thread's exclusive prefix within the CTA (kept for the marking below)
  unsigned long long pre_cta = 0;
  if constexpr (LEAN) {
    unsigned long long x = qs;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    unsigned long long wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NTR / 32; ++w) {
      const unsigned long long y = s_w[w];
      if (w < warp) wpre += y;
      tot += y;
    }
    pre_cta = wpre + (x - qs);
    qs = tot;
  } else {
    qs = block_sum_u64<NTR>(qs, s_w);
    if (ess_rule) {
      e1 = block_sum_u64<NTR>(e1, s_w);
      e2 = block_sum_u64<NTR>(e2, s_w);
    }
  }
  if (threadIdx.x == 0) {
    s_pub_q = qs;
    s_pub_e[0] = e1;
    s_pub_e[1] = e2;
  }
  cl.sync();
  unsigned long long Sb = 0, Q = 0, E1 = 0, E2 = 0;
  for (int r = 0; r < C; ++r) {
    const unsigned long long x = *cl.map_shared_rank(&s_pub_q, r);
    if (r < rank) Sb += x;
    Q += x;
    if (ess_rule) {
      E1 += *cl.map_shared_rank(&s_pub_e[0], r);
      E2 += *cl.map_shared_rank(&s_pub_e[1], r);
    }
  }
  // Alg. 1: resample only when N_eff < N_thresh (every CTA of the cluster
  // decides alike from the same sums)
  const bool resample = !ess_rule || Q == 0 || ess_below(E1, E2, (uint32_t)Np, Pt->ess_t);
  // No more reads of the other CTAs' shared memory: arrive now, wait (so
  // that this CTA's shared memory outlives their reads) only at the end.
  // LEAN: the CTAs write each other's mark arrays below, and a whole
  // cluster barrier follows.
  if constexpr (!LEAN) cluster_arrive();

  // Rank 0 reports the group's weight (M, Q) and resampling decision, which
  // is all the track's global step reads, and takes the group's ticket; the
  // group estimate and ESS follow.  A ticket per track counts the groups
  // that have reported: the track's global step runs once all G have, on
  // the extra cluster of a one-track launch, else on the last taker (its
  // rank-0 CTA, before its own ancestors, so that the global step overlaps
  // the other groups' work).  The reporting thread fences before its
  // ticket; the last taker fences before the reads.  The ancestors are not
  // among the global step's inputs.
  if (rank == 0) {
    GroupState& G = a.gs[grp];
    if (threadIdx.x == 0) {
      G.M = M;
      G.Q = Q;
      G.carry_next = resample ? 0 : 1;
      if (a.fuse_global == 2) {
        __threadfence();
        atomicAdd(&a.glob.ts[d.track].ticket, 1u);
      }
    }
    if (a.fuse_global == 1) {
      __shared__ int s_last;
      if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.glob.ts[d.track].ticket, 1u);
        s_last = (prev + 1u == (unsigned)a.glob.trk[d.track].G) ? 1 : 0;
        __threadfence();
      }
      __syncthreads();
      if (s_last) {
        global_step_call<NTR>(a.glob, d.track, *reinterpret_cast<GlobalScratch*>(s_dyn_rs));
        if (threadIdx.x == 0) a.glob.ts[d.track].ticket = 0u;
        __syncthreads();  // the scratch is the prefix array below
      }
    }
    // group estimate and ESS from the propagate tiles' partial sums, each
    // tile's sums rescaled from its own maximum to the group maximum
    if (a.tile_part != nullptr) {
      float acc[7] = {0, 0, 0, 0, 0, 0, 0};
      if (Q != 0) {
        for (int t = threadIdx.x; t < d.tile_count; t += NTR) {
          const float* tp = a.tile_part + (long long)(d.tile_begin + t) * 8;
          const float Mt = tp[0];
          if (!(Mt - M >= -87.0f)) continue;
          const float sc = __expf(Mt - M);
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[q] = fmaf(sc, tp[1 + q], acc[q]);
          acc[6] = fmaf(sc * sc, tp[7], acc[6]);
        }
      }
#pragma unroll
      for (int q = 0; q < 7; ++q) acc[q] = warp_sum(acc[q]);
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 7; ++q) s_stat[warp][q] = acc[q];
      __syncthreads();
      if (threadIdx.x == 0) {
        float t7[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < NTR / 32; ++w)
          for (int q = 0; q < 7; ++q) t7[q] += s_stat[w][q];
        const bool ok = (Q != 0) && t7[0] > 0.0f;
        for (int q = 0; q < 5; ++q) G.xs[q] = ok ? t7[1 + q] / t7[0] : 0.0f;
        G.ess = ok ? t7[0] * t7[0] / t7[6] : 0.0f;
      }
    }
  }

  const unsigned long long obase = a.local_idx ? 0ull : (unsigned long long)(d.g) * (unsigned long long)Np;
  uint32_t* __restrict__ anc = a.anc + (kk & 1) * a.anc_stride + d.base;
  if (Q == 0 || !resample) {
    // no finite weight, or Alg. 1's test keeps the particles: identity
    for (int i = lo + threadIdx.x; i < hi; i += NTR) {
      anc[i] = (uint32_t)(obase + i);
      if (!LEAN && a.q_out) a.q_out[d.base + i] = 0ull;
    }
  } else {
    // the threshold constants, with the track's precomputed reciprocal of Np
    // when it has one: every thread's own (LEAN), else one thread's for the
    // CTA
    Thresholds th;
    if constexpr (LEAN) {
      if (Pt)
        th.init_magic(Q, (uint32_t)Np, u, Pt->m_Np);
      else
        th.init(Q, (uint32_t)Np, u);
    } else {
      if (threadIdx.x == 0) {
        if (a.glob.trk)
          s_th.init_magic(Q, (uint32_t)Np, u, a.glob.trk[d.track].m_Np);
        else
          s_th.init(Q, (uint32_t)Np, u);
      }
      __syncthreads();
      th = s_th;
    }
    const float inv_Q = 1.0f / u64_to_float_approx(Q);
    if constexpr (LEAN) {
      // Alg. 3 step 7 by marking: item i takes the outputs O_i .. O_{i+1} - 1,
      // O_i = #{j : T_j < S_i} with S_i the sum of the codes before it.  An
      // item with outputs writes i + 1 at position O_i, and at the first
      // position of every CTA whose range starts inside its own, into the
      // mark array of the CTA that owns the position (outputs are split over
      // the cluster like items).  A running maximum over each CTA's
      // positions then gives every output its item, with the same work for
      // every CTA however the weight is spread.
      const int i0 = (int)threadIdx.x * RS_ITEMS;
      unsigned long long S = Sb + pre_cta;  // codes before the thread's first item
      const uint32_t mark_addr = (uint32_t)__cvta_generic_to_shared(s_mark);
#ifdef PF_DEBUG
      PF_DBG_INDEX(a.ds, chunk - 1, NTR * RS_ITEMS, 203u);  // the CTA's outputs fit its mark array
#endif
      int c = count_below(th, S, inv_Q, Np, u, a.ds);
#pragma unroll
      for (int r = 0; r < RS_ITEMS; ++r) {
        if (qv[r] == 0ull) continue;
        S += qv[r];
        const int c1 = count_below(th, S, inv_Q, Np, u, a.ds);
        if (c1 > c) {
          const uint32_t item = (uint32_t)(lo + i0 + r) + 1u;
          int own = 0;  // c / chunk (C is at most 16)
          for (int b = 1; b < C; ++b) own += c >= b * chunk ? 1 : 0;
          int pos = c - own * chunk;
#ifdef PF_DEBUG
          own = (int)PF_DBG_INDEX(a.ds, own, C, 201u);
          pos = (int)PF_DBG_INDEX(a.ds, pos, chunk, 202u);
#endif
          sts_cluster_u32(mark_addr + 4u * (uint32_t)pos, (uint32_t)own, item);
          for (int b = own + 1; b * chunk < c1 && b < C; ++b) sts_cluster_u32(mark_addr, (uint32_t)b, item);
        }
        c = c1;
      }
    } else {
    unsigned long long carry = Sb;
    for (int sub = lo; sub < hi; sub += SUB) {
      const int n = min(SUB, hi - sub);
      const int i0 = (int)threadIdx.x * RS_ITEMS;  // first item of this thread (sub-chunk relative)
      if (!single) {
        load_sub(sub);
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) qv[r] = quantize(v[r], M, a.qc);
      }
      if (!LEAN && a.q_out)
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r)
          if (i0 + r < n) a.q_out[d.base + sub + i0 + r] = qv[r];
      // exclusive scan of the thread totals: warp shuffles, then warps
      unsigned long long tsum = 0;
#pragma unroll
      for (int r = 0; r < RS_ITEMS; ++r) tsum += qv[r];
      unsigned long long x = tsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
      }
      if (lane == 31) s_w[warp] = x;
      __syncthreads();
      unsigned long long wpre = 0, tot = 0;
#pragma unroll
      for (int w = 0; w < NTR / 32; ++w) {
        const unsigned long long y = s_w[w];
        if (w < warp) wpre += y;
        tot += y;
      }
      // inclusive prefixes of the items (absolute within the group)
      {
        unsigned long long S = carry + wpre + (x - tsum);
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
          S += qv[r];
          s_incl[pad8(i0 + r)] = S;
        }
      }
      if (threadIdx.x == 0) {
        s_jlo = count_below(th, carry, inv_Q, Np, u, a.ds);
        s_jhi = count_below(th, carry + tot, inv_Q, Np, u, a.ds);
      }
      __syncthreads();
      merge_windows<NTR>(s_incl, s_out, s_th, s_jlo, s_jhi, n, obase + sub, anc);
      carry += tot;
      __syncthreads();
    }
    }
  }

  if constexpr (LEAN) {
    cl.sync();  // every mark has landed, and the reads of s_pub_q are done
    if (Q != 0 && resample) {
      // running maximum over this CTA's positions p0 + 0 .. n_out - 1 (its
      // first position always holds a mark)
      const int p0 = rank * chunk, n_out = min(chunk, Np - p0);
      const int i0 = (int)threadIdx.x * RS_ITEMS;
      const uint4 m0 = reinterpret_cast<const uint4*>(s_mark)[2 * threadIdx.x];
      const uint4 m1 = reinterpret_cast<const uint4*>(s_mark)[2 * threadIdx.x + 1];
      uint32_t m[RS_ITEMS] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
      for (int r = 1; r < RS_ITEMS; ++r) m[r] = max(m[r], m[r - 1]);
      uint32_t x = m[RS_ITEMS - 1];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = max(x, t);
      }
      uint32_t pre = __shfl_up_sync(0xffffffffu, x, 1);
      if (lane == 0) pre = 0u;
      if (lane == 31) s_w[warp] = x;
      __syncthreads();
#pragma unroll
      for (int w = 0; w < NTR / 32; ++w)
        if (w < warp) pre = max(pre, (uint32_t)s_w[w]);
      if (i0 < n_out && max(pre, m[0]) == 0u) set_error(a.ds, ERR_INVARIANT, 12u, (uint32_t)grp, (uint32_t)(p0 + i0));
      uint32_t o[RS_ITEMS];
#pragma unroll
      for (int r = 0; r < RS_ITEMS; ++r) o[r] = (uint32_t)(obase + max(max(m[r], pre), 1u) - 1u);
      uint32_t* out = anc + p0 + i0;
      if (i0 + RS_ITEMS <= n_out && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        reinterpret_cast<uint4*>(out)[0] = make_uint4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<uint4*>(out)[1] = make_uint4(o[4], o[5], o[6], o[7]);
      } else {
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r)
          if (i0 + r < n_out) out[r] = o[r];
      }
    }
  }

  // The next kernel may start once every CTA is past its main work.
  grid_dep_launch();
  if constexpr (!LEAN) cluster_wait();
}



// ============================================================ export helpers
__global__ void k_export_states(const float4* __restrict__ pv, const float* __restrict__ In, long long n,
                                float* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float4 s = pv[i];
    out[i] = s.x;
    out[n + i] = s.y;
    out[2 * n + i] = s.z;
    out[3 * n + i] = s.w;
    out[4 * n + i] = In[i];
  }
}

// ============================================================== launchers
cudaError_t launch_init(const InitArgs& a, int grid, cudaStream_t s) {
  k_init<<<grid, K1_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

// cudaLaunchKernelEx with an optional cluster shape and programmatic
// stream serialization (see launch_* in pf_launch.h).
template <typename... Params, typename Arg>
static cudaError_t launch_ex(void (*kernel)(Params...), dim3 grid, dim3 block, int cluster, bool pdl,
                             cudaStream_t s, const Arg& arg, size_t smem = 0) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int n = 0;
  if (cluster > 0) {
    attr[n].id = cudaLaunchAttributeClusterDimension;
    attr[n].val.clusterDim.x = (unsigned)cluster;
    attr[n].val.clusterDim.y = 1;
    attr[n].val.clusterDim.z = 1;
    ++n;
  }
  if (pdl) {
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  cfg.attrs = attr;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, kernel, arg);
}

cudaError_t launch_frame_prep_table(const FrameTableArgs& a, int blocks_x, bool pdl, cudaStream_t s) {
  return launch_ex(k_frame_prep_table, dim3(blocks_x, a.n_tracks), dim3(256), 0, pdl, s, a);
}

cudaError_t launch_frame_prep(const FrameArgs& a, int nt, int blocks_x, bool pdl, cudaStream_t s) {
  // blocks_x: rows per track (grid-stride)
  return launch_ex(k_frame_prep, dim3(blocks_x, nt), dim3(256), 0, pdl, s, a);
}

template <int R>
static const void* k1_ptr() {
  return (const void*)k_propagate_weight<R, false, false, false>;
}

const void* propagate_kernel(int R) {
  switch (R) {
    case 1: return k1_ptr<1>();
    case 2: return k1_ptr<2>();
    case 3: return k1_ptr<3>();
    case 4: return k1_ptr<4>();
    case 5: return k1_ptr<5>();
    case 6: return k1_ptr<6>();
    case 7: return k1_ptr<7>();
    default: return nullptr;
  }
}

template <int R, bool SINGLE, bool VARIANTS>
static cudaError_t launch_propagate_rs(const K1Args& a, dim3 g, bool pdl, cudaStream_t s) {
  return launch_ex(k_propagate_weight<R, SINGLE, VARIANTS, false>, g, dim3(K1_THREADS), 0, pdl, s, a);
}

template <int R, bool SINGLE, bool VARIANTS>
static cudaError_t launch_fused_rs(const K1Args& a, dim3 g, bool pdl, cudaStream_t s) {
  return launch_ex(k_propagate_weight<R, SINGLE, VARIANTS, true>, g, dim3(K1_THREADS), 0, pdl, s, a, FUSED_SMEM);
}

template <int R>
static cudaError_t launch_fused_r(const K1Args& a, dim3 g, bool pdl, cudaStream_t s) {
  if (a.variants) return launch_fused_rs<R, false, true>(a, g, pdl, s);
  if (a.n_tracks == 1) return launch_fused_rs<R, true, false>(a, g, pdl, s);
  return launch_fused_rs<R, false, false>(a, g, pdl, s);
}

cudaError_t launch_fused_step(const K1Args& a, int R, int grid, bool pdl, cudaStream_t s) {
  const dim3 g(grid);
  switch (R) {
    case 1: return launch_fused_r<1>(a, g, pdl, s);
    case 2: return launch_fused_r<2>(a, g, pdl, s);
    case 3: return launch_fused_r<3>(a, g, pdl, s);
    case 4: return launch_fused_r<4>(a, g, pdl, s);
    case 5: return launch_fused_r<5>(a, g, pdl, s);
    case 6: return launch_fused_r<6>(a, g, pdl, s);
    case 7: return launch_fused_r<7>(a, g, pdl, s);
    default: return cudaErrorInvalidValue;
  }
}

// Resident fused-step CTAs per SM (the single-track instance of radius R;
// the instances differ little in registers).
cudaError_t fused_occupancy(int R, int* blocks_per_sm) {
  const void* f = nullptr;
  switch (R) {
    case 1: f = (const void*)k_propagate_weight<1, true, false, true>; break;
    case 2: f = (const void*)k_propagate_weight<2, true, false, true>; break;
    case 3: f = (const void*)k_propagate_weight<3, true, false, true>; break;
    case 4: f = (const void*)k_propagate_weight<4, true, false, true>; break;
    case 5: f = (const void*)k_propagate_weight<5, true, false, true>; break;
    case 6: f = (const void*)k_propagate_weight<6, true, false, true>; break;
    case 7: f = (const void*)k_propagate_weight<7, true, false, true>; break;
    default: return cudaErrorInvalidValue;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, K1_THREADS, FUSED_SMEM);
}

// Instances: one track, several tracks, and tracks that use a method
// variant (groups that carry their particles' own weights under Alg. 1's
// resampling test, or keyed send sets; any track count, frames prepared).
template <int R>
static cudaError_t launch_propagate_r(const K1Args& a, dim3 g, bool pdl, cudaStream_t s) {
  if (a.variants) return launch_propagate_rs<R, false, true>(a, g, pdl, s);
  if (a.n_tracks == 1) return launch_propagate_rs<R, true, false>(a, g, pdl, s);
  return launch_propagate_rs<R, false, false>(a, g, pdl, s);
}

cudaError_t launch_propagate(const K1Args& a, int R, int grid, bool pdl, cudaStream_t s) {
  const dim3 g(grid);
  switch (R) {
    case 1: return launch_propagate_r<1>(a, g, pdl, s);
    case 2: return launch_propagate_r<2>(a, g, pdl, s);
    case 3: return launch_propagate_r<3>(a, g, pdl, s);
    case 4: return launch_propagate_r<4>(a, g, pdl, s);
    case 5: return launch_propagate_r<5>(a, g, pdl, s);
    case 6: return launch_propagate_r<6>(a, g, pdl, s);
    case 7: return launch_propagate_r<7>(a, g, pdl, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int NTR, bool LEAN>
static cudaError_t launch_resample_t(const ResampleArgs& a, int n_groups, int cluster, bool pdl, cudaStream_t s) {
  constexpr size_t smem = LEAN ? RS_MARK_OFF + NTR * RS_ITEMS * sizeof(uint32_t)
                              : pad8(NTR * RS_ITEMS) * sizeof(unsigned long long) +
                                    pad8(2 * NTR * RS_ITEMS) * sizeof(uint32_t);
  static_assert(sizeof(GlobalScratch) <= smem, "the global step's scratch lives in the resampler's shared memory");
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_resample<NTR, LEAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const int clusters = n_groups + (a.fuse_global == 2 ? 1 : 0);  // the global step's extra cluster
  return launch_ex(k_resample<NTR, LEAN>, dim3((unsigned)(clusters * cluster)), dim3(NTR), cluster, pdl, s, a, smem);
}

cudaError_t launch_resample(const ResampleArgs& a, int n_groups, int cluster, bool pdl, cudaStream_t s, int threads) {
  const long long chunk = (((long long)a.max_np + cluster - 1) / cluster + 7) / 8 * 8;  // as in k_resample
  if (a.lean && !a.q_out && chunk <= (long long)threads * RS_ITEMS) {
    if (threads == RS_THREADS_SMALL) return launch_resample_t<RS_THREADS_SMALL, true>(a, n_groups, cluster, pdl, s);
    return launch_resample_t<RS_THREADS, true>(a, n_groups, cluster, pdl, s);
  }
  if (threads == RS_THREADS_SMALL) return launch_resample_t<RS_THREADS_SMALL, false>(a, n_groups, cluster, pdl, s);
  return launch_resample_t<RS_THREADS, false>(a, n_groups, cluster, pdl, s);
}

cudaError_t launch_global(const GlobalArgs& a, int n_tracks, cudaStream_t s) {
  k_global<<<n_tracks, GL_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finish(const GlobalArgs& a, int n_tracks, cudaStream_t s) {
  k_finish<<<n_tracks, K1_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finish_out(const GlobalArgs& a, int n_tracks, float* xhat, double* logZ, bool pdl,
                              cudaStream_t s) {
  return launch_ex(k_finish_out, dim3(n_tracks), dim3(K1_THREADS), 0, pdl, s, FinishOutArgs{a, xhat, logZ});
}

cudaError_t launch_export_states(const float4* pv, const float* In, long long n, float* out, cudaStream_t s) {
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_export_states<<<grid > 0 ? grid : 1, 256, 0, s>>>(pv, In, n, out);
  return cudaGetLastError();
}

cudaError_t k1_occupancy(int R, int* blocks_per_sm) {
  const void* f = propagate_kernel(R);
  if (!f) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, K1_THREADS, 0);
}

}  // namespace pf
