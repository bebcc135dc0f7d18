// pf_kernels.cu -- CUDA kernels (sm_103a) of one RNA / ARNA filter step.
//
// Paper: Demirel et al., "An Adaptive Distributed Resampling Algorithm with
// Non-Proportional Allocation" (arXiv:1310.4624).
//
// One step k of Alg. 3 (Alg. 2 for RNA) is four launches on one stream:
//   k_frame_prep        y = z - b into a zero-padded frame (Sec. V model)
//   k_propagate_weight  ring exchange composed with the previous resampling
//                       (Alg. 3 steps 3-4), propagation (Alg. 1 step P),
//                       likelihood (step U) and per-tile partial sums for
//                       the group estimate (Alg. 3 step 6)
//   k_resample          per-group exact systematic resampling on fixed-point
//                       weight codes (Alg. 3 step 7), one thread-block
//                       cluster per group, partial sums exchanged through
//                       distributed shared memory
//   k_global            per track: the master PE's reduction (steps 9-10),
//                       S10 weight carry (step 8), and the ring order
//                       (step 1) and exchange count (step 2, Eq. 3/4) of the
//                       next step
// The step index lives on the device, so the same launch sequence serves
// every step.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pf_device.cuh"
#include "pf_launch.h"

namespace cg = cooperative_groups;

namespace pf {

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide reductions; every thread gets the result.  `sh` holds one slot
// per warp and is free again on return.
template <int NT>
__device__ __forceinline__ float block_max(float v, float* sh) {
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = sh[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) r = fmaxf(r, sh[w]);
  __syncthreads();
  return r;
}
template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) r += sh[w];
  __syncthreads();
  return r;
}
template <int NT>
__device__ __forceinline__ double block_max_d(double v, double* sh) {
  v = warp_max_d(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) r = fmax(r, sh[w]);
  __syncthreads();
  return r;
}
template <int NT>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sh) {
  v = warp_sum_u64(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long r = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) r += sh[w];
  __syncthreads();
  return r;
}

// ===================================================================== K0
// Initial population (Sec. V tracking / information-sharing modes), drawn
// from Philox stream INIT into the buffer step 0 reads.
__global__ void __launch_bounds__(K1_THREADS) k_init(InitArgs a) {
  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int4 td = a.tiles[tile];
    if ((int)threadIdx.x >= td.w) continue;
    const TrackParams& P = a.trk[td.x];
    const int g = td.y, j = td.z + threadIdx.x;
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

// ===================================================================== K8
// y = z - b into the interior of the zero-padded frame; the padding (2R+1
// pixels on each side, zeroed once at init) stands for "outside the image
// counts as background".
__global__ void k_frame_prep(FrameArgs a) {
  const int tt = blockIdx.y;
  const TrackParams& P = a.trk[a.t0 + tt];
  const float* __restrict__ z = a.frames[tt];
  float* __restrict__ yp = a.ypad + P.ypad_off;
  const int pad = 2 * a.R + 1;
  const long long n = (long long)P.H * P.W;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(p / P.W), u = (int)(p - (long long)v * P.W);
    yp[(long long)(v + pad) * P.pitch + (u + pad)] = __fsub_rn(__ldg(z + p), P.bg);
  }
}

// ===================================================================== K1
// Log-likelihood of one particle (Sec. V appearance model):
//   -sum_{(2R+1)^2 patch} (y - I gx(u) gy(v))^2 / (2 sigma_obs^2),
// patch centred on the nearest pixel, y = z - b, y = 0 outside the frame.
// Reads the padded frame; the centre is clamped so that a patch entirely
// off the frame reads padding, while the model terms use the true centre.
template <int R>
__device__ __forceinline__ float loglik(const float* __restrict__ yp, int pitch, int H, int W, float x, float y,
                                        float I, float c_psf, float inv2so2) {
  constexpr int D = 2 * R + 1;
  constexpr int PAD = 2 * R + 1;
  const float cxf = floorf(x + 0.5f), cyf = floorf(y + 0.5f);
  const int cx = (int)fminf(fmaxf(cxf, -(float)(R + 1)), (float)(W + R));
  const int cy = (int)fminf(fmaxf(cyf, -(float)(R + 1)), (float)(H + R));
  const float* __restrict__ row = yp + (long long)(cy - R + PAD) * pitch + (cx - R + PAD);
  float gxI[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float d = (cxf + (float)(a - R)) - x;
    gxI[a] = I * ex2(-c_psf * d * d);
  }
  float acc = 0.0f;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    const float d = (cyf + (float)(b - R)) - y;
    const float gy = ex2(-c_psf * d * d);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float r = fmaf(-gxI[a], gy, __ldg(row + a));
      acc = fmaf(r, r, acc);
    }
    row += pitch;
  }
  return -acc * inv2so2;
}

// Slot i = (group g, slot j) of step k takes the particle of slot src of the
// exchanged population (Sec. III-A/C): group g's send set is the systematic
// slot subsample s_{g,t} = floor((t Np + o_g) / N_ex); slot s_{r,t} of the
// receiver r gets sender pred(r)'s slot s_{pred(r),t} with its origin
// weight.  Returns the origin group.
__device__ __forceinline__ int exchange_source(const GroupState* __restrict__ gs, int g, int j, int Np, int nex,
                                               long long& src_local) {
  src_local = (long long)g * Np + j;
  if (nex <= 0) return g;
  const long long o_r = gs[g].exo;
  const long long num = (long long)j * nex - o_r;
  const long long t = num <= 0 ? 0 : (num + Np - 1) / Np;
  if (t < nex && t * Np + o_r < (long long)(j + 1) * nex) {
    const int sg = gs[g].pred;
    const long long o_s = gs[sg].exo;
    src_local = (long long)sg * Np + (t * Np + o_s) / nex;
    return sg;
  }
  return g;
}

template <int R>
__global__ void __launch_bounds__(K1_THREADS) k_propagate_weight(K1Args a) {
  const int k = a.ts[0].k;
  const float4* __restrict__ pv_prev = (k & 1) ? a.pv0 : a.pv1;
  const float* __restrict__ I_prev = (k & 1) ? a.I0 : a.I1;
  float4* __restrict__ pv_cur = (k & 1) ? a.pv1 : a.pv0;
  float* __restrict__ I_cur = (k & 1) ? a.I1 : a.I0;
  __shared__ float s_red[K1_THREADS / 32][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int4 td = a.tiles[tile];
    const TrackParams& P = a.trk[td.x];
    const bool active = (int)threadIdx.x < td.w;
    float lw = -INFINITY, I = 0.0f;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) {
      const int g = td.y, j = td.z + threadIdx.x, Np = P.Np;
      const long long il = (long long)g * Np + j;
      const GroupState* __restrict__ gs = a.grp + P.group_off;
      long long src;
      const int og = (k == 0) ? g : exchange_source(gs, g, j, Np, a.ts[td.x].n_ex, src);
      if (k == 0) src = il;
      const long long par = (k == 0) ? src : (long long)a.anc[P.part_off + src];
      if (par < 0 || par >= (long long)P.G * Np) {
        set_error(a.ds, ERR_INDEX, 1u, (uint32_t)tile, (uint32_t)par);
      } else {
        s = pv_prev[P.part_off + par];
        I = I_prev[P.part_off + par];
      }
      if (k > 0) {
        // Alg. 1 step P: nearly constant velocity, unit frame interval
        const uint4 w0 = philox(P.key0, P.key1, make_uint4(j, g, k, P.tag | (ST_PROP << 4) | 0u));
        const uint4 w1 = philox(P.key0, P.key1, make_uint4(j, g, k, P.tag | (ST_PROP << 4) | 1u));
        float e0, e1, e2, e3, e4, e5;
        box_muller(w0.x, w0.y, e0, e1);
        box_muller(w0.z, w0.w, e2, e3);
        box_muller(w1.x, w1.y, e4, e5);
        s.x = fmaf(P.spos, e0, s.x + s.z);
        s.y = fmaf(P.spos, e1, s.y + s.w);
        s.z = fmaf(P.sv, e2, s.z);
        s.w = fmaf(P.sv, e3, s.w);
        I = fmaf(P.sI, e4, I);
      }
      const long long i = P.part_off + il;
      pv_cur[i] = s;
      I_cur[i] = I;
      if (P.record) a.parent[P.parent_off + (long long)(k % a.history) * ((long long)P.G * Np) + il] = (uint32_t)par;
      // Alg. 1 step U with the renormalised carried weight (Alg. 3 step 4)
      lw = gs[og].off + loglik<R>(a.ypad + P.ypad_off, P.pitch, P.H, P.W, s.x, s.y, I, P.c_psf, P.inv2so2);
      a.lw[i] = lw;
    }
    // Per-tile partial sums for the group estimate, relative to the tile max.
    float m = warp_max(active ? lw : -INFINITY);
    if (lane == 0) s_red[warp][0] = m;
    __syncthreads();
    float Mt = s_red[0][0];
#pragma unroll
    for (int w = 1; w < K1_THREADS / 32; ++w) Mt = fmaxf(Mt, s_red[w][0]);
    __syncthreads();
    const float e = (active && lw - Mt >= -87.0f) ? __expf(lw - Mt) : 0.0f;
    float v[7] = {e, e * s.x, e * s.y, e * s.z, e * s.w, e * I, e * e};
#pragma unroll
    for (int q = 0; q < 7; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 7; ++q) s_red[warp][q + 1] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      float r;
      if (threadIdx.x == 0) {
        r = Mt;
      } else {
        r = 0.0f;
#pragma unroll
        for (int w = 0; w < K1_THREADS / 32; ++w) r += s_red[w][threadIdx.x];
      }
      a.tile_part[(long long)tile * 8 + threadIdx.x] = r;
    }
    __syncthreads();
  }
}

// ===================================================================== K3
// Number of outputs j in [0, Np) with (j 2^32 + u) Q < S Np 2^32: an FP32
// estimate, then exact 128-bit corrections (the estimate is within 1).
__device__ __forceinline__ long long count_below(const ThetaCmp& th, unsigned long long S, int Np, DevState* ds) {
  if (S == 0) return 0;
  const float est = __fdividef(__ull2float_rn(S), __ull2float_rn(th.Q)) * (float)Np - (float)th.u * 2.3283064365386963e-10f;
  long long c = (long long)ceilf(fminf(fmaxf(est, 0.0f), (float)Np));
  int it = 0;
  while (c < Np && th.below(c, S) && it < 64) { ++c; ++it; }
  while (c > 0 && !th.below(c - 1, S) && it < 64) { --c; ++it; }
  if (it >= 64) set_error(ds, ERR_INVARIANT, 3u, (uint32_t)S, (uint32_t)c);
  return c;
}

__global__ void __launch_bounds__(RS_THREADS) k_resample(ResampleArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int grp = blockIdx.x / C;
  const GroupDesc d = a.gd[grp];
  const int Np = d.Np;
  const int chunk = (Np + C - 1) / C;
  const int lo = min(rank * chunk, Np), hi = min(lo + chunk, Np);
  const float* __restrict__ lw = a.lw + d.base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  __shared__ float s_pub_max;
  __shared__ unsigned long long s_pub_q;
  __shared__ float s_f[RS_THREADS / 32];
  __shared__ double s_d[RS_THREADS / 32];
  __shared__ unsigned long long s_w[RS_THREADS / 32];
  __shared__ unsigned long long s_incl[RS_SUB];

  // group maximum over the cluster
  float m = -INFINITY;
  for (int i = lo + threadIdx.x; i < hi; i += RS_THREADS) m = fmaxf(m, lw[i]);
  m = block_max<RS_THREADS>(m, s_f);
  if (threadIdx.x == 0) s_pub_max = m;
  cl.sync();
  float M = -INFINITY;
  for (int r = 0; r < C; ++r) M = fmaxf(M, *cl.map_shared_rank(&s_pub_max, r));

  // this CTA's total weight code, then the cluster prefix and group total
  unsigned long long qs = 0;
  for (int i = lo + threadIdx.x; i < hi; i += RS_THREADS) qs += quantize(lw[i], M, a.qc);
  qs = block_sum_u64<RS_THREADS>(qs, s_w);
  if (threadIdx.x == 0) s_pub_q = qs;
  cl.sync();
  unsigned long long Sb = 0, Q = 0;
  for (int r = 0; r < C; ++r) {
    const unsigned long long v = *cl.map_shared_rank(&s_pub_q, r);
    if (r < rank) Sb += v;
    Q += v;
  }

  const uint32_t u = a.u_arr ? a.u_arr[grp] : a.gs[grp].u;
  const unsigned long long obase = a.local_idx ? 0ull : (unsigned long long)(d.g) * (unsigned long long)Np;
  uint32_t* __restrict__ anc = a.anc + d.base;
  if (Q == 0) {
    // no finite weight: identity
    for (int i = lo + threadIdx.x; i < hi; i += RS_THREADS) {
      anc[i] = (uint32_t)(obase + i);
      if (a.q_out) a.q_out[d.base + i] = 0ull;
    }
  } else {
    const ThetaCmp th{Q, (unsigned long long)Np, u};
    unsigned long long carry = Sb;
    for (int sub = lo; sub < hi; sub += RS_SUB) {
      const int n = min(RS_SUB, hi - sub);
      // warp-segmented inclusive scan: warp w owns items [w*32*RS_ITEMS, ...)
      unsigned long long run = 0;
#pragma unroll
      for (int r = 0; r < RS_ITEMS; ++r) {
        const int it = warp * (32 * RS_ITEMS) + r * 32 + lane;
        unsigned long long q = 0;
        if (it < n) {
          q = quantize(lw[sub + it], M, a.qc);
          if (a.q_out) a.q_out[d.base + sub + it] = q;
        }
        unsigned long long v = q;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += t;
        }
        s_incl[it] = run + v;
        run += __shfl_sync(0xffffffffu, v, 31);
      }
      if (lane == 0) s_w[warp] = run;
      __syncthreads();
      unsigned long long wpre = 0, tot = 0;
#pragma unroll
      for (int w = 0; w < RS_THREADS / 32; ++w) {
        const unsigned long long v = s_w[w];
        if (w < warp) wpre += v;
        tot += v;
      }
#pragma unroll
      for (int r = 0; r < RS_ITEMS; ++r) s_incl[warp * (32 * RS_ITEMS) + r * 32 + lane] += carry + wpre;
      __syncthreads();
      // outputs whose ancestor lies in this sub-chunk: binary search for the
      // first item whose inclusive prefix exceeds the output's threshold
      const long long jlo = count_below(th, carry, Np, a.ds);
      const long long jhi = count_below(th, carry + tot, Np, a.ds);
      for (long long j = jlo + threadIdx.x; j < jhi; j += RS_THREADS) {
        const U128 lhs = mul64(((unsigned long long)j << 32) | u, Q);
        int L = 0, Hh = n - 1;
        while (L < Hh) {
          const int mid = (L + Hh) >> 1;
          if (lt128(lhs, shl32(mul64(s_incl[mid], (unsigned long long)Np)))) Hh = mid;
          else L = mid + 1;
        }
        anc[j] = (uint32_t)(obase + sub + L);
      }
      carry += tot;
      __syncthreads();
    }
  }

  // group estimate and ESS from the propagate tiles' partial sums (rank 0)
  if (rank == 0) {
    GroupState& G = a.gs[grp];
    if (a.tile_part != nullptr) {
      double acc[7] = {0, 0, 0, 0, 0, 0, 0};
      if (Q != 0) {
        for (int t = threadIdx.x; t < d.tile_count; t += RS_THREADS) {
          const float* tp = a.tile_part + (long long)(d.tile_begin + t) * 8;
          const float Mt = tp[0];
          if (!(Mt - M >= -87.0f)) continue;
          const double sc = exp((double)Mt - (double)M);
          for (int q = 0; q < 6; ++q) acc[q] += sc * (double)tp[1 + q];
          acc[6] += sc * sc * (double)tp[7];
        }
      }
      for (int q = 0; q < 7; ++q) acc[q] = block_sum_d<RS_THREADS>(acc[q], s_d);
      if (threadIdx.x == 0) {
        const bool ok = (Q != 0) && acc[0] > 0.0;
        for (int q = 0; q < 5; ++q) G.xs[q] = ok ? (float)(acc[1 + q] / acc[0]) : 0.0f;
        G.ess = ok ? (float)(acc[0] * acc[0] / acc[6]) : 0.0f;
      }
    }
    if (threadIdx.x == 0) {
      G.M = M;
      G.Q = Q;
    }
  }
  cl.sync();  // keep shared memory alive until every CTA has read it
}

// ===================================================================== K5
// Per track: the master PE's reduction (Alg. 3 steps 9-10) and weight carry
// (step 8) for step k, then ring order (step 1) and exchange count (step 2)
// for step k+1.  FP64 throughout: it is G-sized.
__global__ void __launch_bounds__(GL_THREADS) k_global(GlobalArgs a) {
  const int t = blockIdx.x;
  const TrackParams& P = a.trk[t];
  TrackState* T = a.ts + t;
  GroupState* gs = a.gs + P.group_off;
  int* ring = a.ring + P.group_off;
  const int G = P.G;
  const int k = T->k;
  const double LN2 = 0.69314718055994530942;
  __shared__ double s_d[GL_THREADS / 32];
  __shared__ int s_ring[MAX_G];
  __shared__ uint32_t s_r[MAX_G];
  __shared__ int s_deg;
  __shared__ double s_logc;

  if (a.finalize) {
    // S7 -> S8: Lambda'_m = M_m + ln(Q_m 2^-40); log c_k = LSE Lambda'
    double lmax = -INFINITY;
    int deg = 0;
    for (int m = threadIdx.x; m < G; m += GL_THREADS) {
      const unsigned long long Q = gs[m].Q;
      const double lam = (Q != 0) ? (double)gs[m].M + log((double)Q) - 40.0 * LN2 : -INFINITY;
      gs[m].lambda = lam;
      lmax = fmax(lmax, lam);
      deg += (Q == 0);
    }
    lmax = block_max_d<GL_THREADS>(lmax, s_d);
    deg = (int)block_sum_d<GL_THREADS>((double)deg, s_d);
    double sw = 0.0;
    if (isfinite(lmax))
      for (int m = threadIdx.x; m < G; m += GL_THREADS) sw += exp(gs[m].lambda - lmax);
    sw = block_sum_d<GL_THREADS>(sw, s_d);
    const double logc = isfinite(lmax) ? lmax + log(sw) : -INFINITY;
    double xh[5];
    for (int q = 0; q < 5; ++q) {
      double acc = 0.0;
      if (isfinite(logc))
        for (int m = threadIdx.x; m < G; m += GL_THREADS)
          if (gs[m].Q != 0) acc += exp(gs[m].lambda - logc) * (double)gs[m].xs[q];
      xh[q] = block_sum_d<GL_THREADS>(acc, s_d);
    }
    const int hslot = k % a.history;
    for (int m = threadIdx.x; m < G; m += GL_THREADS) {
      GroupHist& gh = a.ghist[P.ghist_off + (long long)hslot * G + m];
      gh.ring = ring[m];
      gh.logW = gs[m].lambda;
      for (int q = 0; q < 5; ++q) gh.xs[q] = gs[m].xs[q];
      gh.ess = gs[m].ess;
    }
    if (threadIdx.x == 0) {
      T->log_c = logc;
      T->log_Z += logc;
      for (int q = 0; q < 5; ++q) T->xhat[q] = (float)xh[q];
      T->degenerate = deg;
      if (deg == G) T->flags |= 1;
      T->steps_done = k + 1;
      HistRec& h = a.hist[P.hist_off + hslot];
      h.step = k;
      h.n_ex = T->n_ex;
      h.pe_eff = T->pe_eff;
      h.log_c = logc;
      h.log_Z = T->log_Z;
      for (int q = 0; q < 5; ++q) h.xhat[q] = (float)xh[q];
      h.degenerate = deg;
      s_deg = deg;
    }
    __syncthreads();
    if (s_deg == G)  // every group lost its weight: restart from equal weights
      for (int m = threadIdx.x; m < G; m += GL_THREADS) gs[m].lambda = 0.0;
  } else {
    for (int m = threadIdx.x; m < G; m += GL_THREADS) gs[m].lambda = 0.0;
  }
  __syncthreads();

  const int k1 = a.finalize ? k + 1 : 0;
  // Eq. 4 from the carried weights; LSE for the renormalisation (step 4)
  double lmax = -INFINITY;
  for (int m = threadIdx.x; m < G; m += GL_THREADS) lmax = fmax(lmax, gs[m].lambda);
  lmax = block_max_d<GL_THREADS>(lmax, s_d);
  double sw = 0.0, sw2 = 0.0;
  for (int m = threadIdx.x; m < G; m += GL_THREADS) {
    const double w = exp(gs[m].lambda - lmax);
    sw += w;
    sw2 += w * w;
  }
  sw = block_sum_d<GL_THREADS>(sw, s_d);
  sw2 = block_sum_d<GL_THREADS>(sw2, s_d);
  const double pe = sw * sw / sw2;
  const double lse = lmax + log(sw);
  if (threadIdx.x == 0) s_logc = lse;

  // ring order for step k1 (Sec. IV-B): Fisher-Yates on the identity
  const bool shuffle = (P.mode == MODE_ARNA) && k1 >= 1 && G > 1;
  for (int p = threadIdx.x; p < G; p += GL_THREADS) {
    s_ring[p] = p;
    if (shuffle && p >= 1) {
      uint32_t r;
      if (!draw_bounded(P.key0, P.key1, P.tag, ST_RING, (uint32_t)p, (uint32_t)k1, (uint32_t)p + 1u, r))
        set_error(a.ds, ERR_DRAW, 1u, (uint32_t)t, (uint32_t)p);
      s_r[p] = r;
    }
  }
  __syncthreads();
  if (shuffle && threadIdx.x == 0) {
    for (int j = G - 1; j >= 1; --j) {
      const int r = (int)s_r[j];
      const int tmp = s_ring[j];
      s_ring[j] = s_ring[r];
      s_ring[r] = tmp;
    }
  }
  __syncthreads();

  // exchange count for step k1 (Eq. 3 with the Sec. V-A cut-off)
  int nex = 0;
  if (k1 >= 1 && G > 1) {
    double rho;
    if (P.mode == MODE_ARNA) {
      if (!(pe < (double)P.cutoff * (double)G)) {
        rho = 0.0;
      } else {
        rho = 0.5 - 0.5 * (pe - 1.0) / (double)(G - 1);
        rho = fmin(fmax(rho, 0.0), 0.5);
      }
    } else {
      rho = fmin(fmax((double)P.ex_ratio, 0.0), 1.0);
    }
    nex = (int)floor(rho * (double)P.Np);
  }
  const double lnNp = log((double)P.Np);
  for (int p = threadIdx.x; p < G; p += GL_THREADS) {
    ring[p] = s_ring[p];
    gs[s_ring[p]].pred = s_ring[(p + G - 1) % G];
    uint32_t o = 0;
    if (nex > 0 && !draw_bounded(P.key0, P.key1, P.tag, ST_EXCH, (uint32_t)p, (uint32_t)k1, (uint32_t)P.Np, o))
      set_error(a.ds, ERR_DRAW, 2u, (uint32_t)t, (uint32_t)p);
    gs[p].exo = o;
    gs[p].u = philox(P.key0, P.key1, make_uint4((uint32_t)p, 0u, (uint32_t)k1, P.tag | (ST_RESAMPLE << 4))).x;
    gs[p].off = (float)(gs[p].lambda - lnNp - s_logc);
  }
  if (threadIdx.x == 0) {
    T->n_ex = nex;
    T->pe_eff = pe;
    T->k = k1;
  }
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

cudaError_t launch_frame_prep(const FrameArgs& a, int nt, int blocks_x, cudaStream_t s) {
  k_frame_prep<<<dim3(blocks_x, nt), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <int R>
static const void* k1_ptr() {
  return (const void*)k_propagate_weight<R>;
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

cudaError_t launch_propagate(const K1Args& a, int R, int grid, cudaStream_t s) {
  switch (R) {
    case 1: k_propagate_weight<1><<<grid, K1_THREADS, 0, s>>>(a); break;
    case 2: k_propagate_weight<2><<<grid, K1_THREADS, 0, s>>>(a); break;
    case 3: k_propagate_weight<3><<<grid, K1_THREADS, 0, s>>>(a); break;
    case 4: k_propagate_weight<4><<<grid, K1_THREADS, 0, s>>>(a); break;
    case 5: k_propagate_weight<5><<<grid, K1_THREADS, 0, s>>>(a); break;
    case 6: k_propagate_weight<6><<<grid, K1_THREADS, 0, s>>>(a); break;
    case 7: k_propagate_weight<7><<<grid, K1_THREADS, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_resample(const ResampleArgs& a, int n_groups, int cluster, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_groups * cluster));
  cfg.blockDim = dim3(RS_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_resample, a);
}

cudaError_t launch_global(const GlobalArgs& a, int n_tracks, cudaStream_t s) {
  k_global<<<n_tracks, GL_THREADS, 0, s>>>(a);
  return cudaGetLastError();
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
