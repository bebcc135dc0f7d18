// pf_adjoint.cu -- kernels of pf_backward: the gradient of log Z = sum_k
// log c_k with respect to theta = (sigma_psf, A, b, sigma_pos, sigma_v) with
// the resampling ancestry of the forward run held fixed.
//
// Paper: Demirel et al., "An Adaptive Distributed Resampling Algorithm with
// Non-Proportional Allocation" (arXiv:1310.4624).  With the ancestry fixed
// the filter (Alg. 3) is a smooth function of theta:
//   X_k(i)   = NCV(X_{k-1}(p_k(i)); theta)            (Alg. 1 step P)
//   lw_k(i)  = lbar_{k-1}(o(i)) - log Np + l_k(i)      (steps 4-5, U)
//   L_k,m    = LSE_{i in m} lw_k(i)                    (step 6)
//   log c_k  = LSE_m L_k,m,  lbar_k = L_k - log c_k    (steps 9-10)
// with o(i) = p_k(i) div Np the origin group of the slot (the exchange puts
// a particle of group o into slot i).  Reverse mode, seed s = d out / d log Z:
//   dL_{T-1,m} = s pi_m,  dL_{k,m} = sum_{i : o_{k+1}(i) = m} dlw_{k+1}(i)
//   dlw_k(i)   = dL_{k,m(i)} exp(lw_k(i) - L_k,m(i))
// (the softmax terms of lbar cancel because sum_m dL_k,m = s at every k);
// states back-propagate through the NCV Jacobian to their recorded parents.
// The forward pass is replayed from the initial population and the recorded
// parents with the same Philox streams; states are recomputed from
// checkpoints, not stored per step.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "pf_device.cuh"
#include "pf_launch.h"
#include "pf_math.cuh"

namespace pf {

// ------------------------------------------------------------------ replay
// Replay of step k for every slot: the state (k >= 1: NCV from the recorded
// parent and the step's normals) and, when weights != 0, the log-weight and
// its per-tile (max, sum exp) for the group log-weights.
template <int R>
__global__ void __launch_bounds__(256) k_replay(ReplayArgs a) {
  constexpr int PAD = 2 * R + 1;
  const int k = a.k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ float s_m[8], s_s[8];
  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int4 td = a.tiles[tile];
    const TrackParams& P = a.trk[td.x];
    const int g = td.y, Np = P.Np;
    const long long Nt = (long long)P.G * Np;
    const int hslot = k % a.history;
    const float log_G = logf((float)P.G), log_Np = logf((float)Np);
    float mx = -INFINITY, sm = 0.0f;
    for (int jj = threadIdx.x; jj < td.w; jj += blockDim.x) {
      const int j = td.z + jj;
      const long long il = (long long)g * Np + j, i = P.part_off + il;
      float4 s;
      float I;
      int o = g;
      if (k >= 1) {
        const long long par = a.parent[P.parent_off + (long long)hslot * Nt + il];
        o = (int)fastdiv((uint32_t)par, P.m_Np);  // origin group (par < 2^31)
        s = a.pv_in[P.part_off + par];
        I = a.I_in[P.part_off + par];
        uint4 w0 = make_uint4(j, g, k, P.tag | (ST_PROP << 4) | 0u);
        uint4 w1 = make_uint4(j, g, k, P.tag | (ST_PROP << 4) | 1u);
        philox2(P.key0, P.key1, w0, w1);
        float e0, e1, e2, e3, e4, e5;
        box_muller_fast(w0.x, w0.y, e0, e1);
        box_muller_fast(w0.z, w0.w, e2, e3);
        box_muller_fast(w1.x, w1.y, e4, e5);
        s.x = fmaf(P.spos, e0, s.x + s.z);
        s.y = fmaf(P.spos, e1, s.y + s.w);
        s.z = fmaf(P.sv, e2, s.z);
        s.w = fmaf(P.sv, e3, s.w);
        I = fmaf(P.sI, e4, I);
        a.pv_out[i] = s;
        a.I_out[i] = I;
      } else {
        s = a.pv_out[i];
        I = a.I_out[i];
      }
      if (a.ck_pv) {
        a.ck_pv[i] = s;
        a.ck_I[i] = I;
      }
      if (a.weights) {
        float gxI[2 * R + 1];
        const float cxf = floorf(s.x + 0.5f), cyf = floorf(s.y + 0.5f);
        gauss_row<R>(cxf, s.x, P.c_psf, P.kappa, gxI);
#pragma unroll
        for (int c = 0; c < 2 * R + 1; ++c) gxI[c] *= I;
        const int pu = (int)fminf(fmaxf(cxf, -(float)(R + 1)), (float)(P.W + R)) - R + PAD;
        const int pv = (int)fminf(fmaxf(cyf, -(float)(R + 1)), (float)(P.H + R)) - R + PAD;
        const float* base = a.ypad + P.ypad_off + (long long)pv * P.pitch + pu;
        const float ss = P.obs_model == 1 ? patch_ss<R, true, false>(base, P.pitch, gxI, cyf - s.y, P.c_psf, P.kappa)
                                          : patch_ss<R, false, false>(base, P.pitch, gxI, cyf - s.y, P.c_psf, P.kappa);
        const float lb = k >= 1 ? (float)a.lbar_prev[P.group_off + o] : -log_G;
        const float lw = lb - log_Np - ss * P.inv2so2;
        if (lw == lw && lw > -INFINITY) {
          if (lw > mx) {
            sm = sm * __expf(mx - lw) + 1.0f;
            mx = lw;
          } else {
            sm += __expf(lw - mx);
          }
        }
      }
    }
    if (a.weights) {
      // block (max, sum exp) of the tile
      float m2 = warp_max(mx);
      float s2 = (mx > -INFINITY) ? sm * __expf(mx - m2) : 0.0f;
      s2 = warp_sum(s2);
      if (lane == 0) {
        s_m[warp] = m2;
        s_s[warp] = s2;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        float M = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = fmaxf(M, s_m[w]);
        float S = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
          if (s_m[w] > -INFINITY) S += s_s[w] * __expf(s_m[w] - M);
        a.tile_part[(long long)tile * 8 + 0] = M;
        a.tile_part[(long long)tile * 8 + 1] = S;
      }
      __syncthreads();
    }
  }
}

// Per track: the replayed group log-weights of step k, log c_k, lbar_k, and
// at the last step the seed of the reverse sweep, dL = s pi.  FP64 (G-sized).
__global__ void __launch_bounds__(256) k_replay_groups(ReplayGroupArgs a) {
  const int t = blockIdx.x;
  const TrackParams& P = a.trk[t];
  const int G = P.G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
  __shared__ double s_lam[MAX_G];
  __shared__ double s_d[32];
  __shared__ double s_lc;
  // L_k,m = LSE over the group's slots, from its tiles' (max, sum exp): a
  // warp per group, its lanes over the tiles
  for (int m = warp; m < G; m += nw) {
    const int t0 = a.gd[P.group_off + m].tile_begin, nt = a.gd[P.group_off + m].tile_count;
    float M = -INFINITY;
    for (int q = lane; q < nt; q += 32) M = fmaxf(M, a.tile_part[(long long)(t0 + q) * 8]);
    M = warp_max(M);
    float S = 0.0f;
    if (M > -INFINITY)
      for (int q = lane; q < nt; q += 32) {
        const float Mt = a.tile_part[(long long)(t0 + q) * 8];
        if (Mt > -INFINITY) S = fmaf(a.tile_part[(long long)(t0 + q) * 8 + 1], expf(Mt - M), S);
      }
    S = warp_sum(S);
    if (lane == 0) s_lam[m] = (M > -INFINITY && S > 0.0f) ? (double)M + log((double)S) : -INFINITY;
  }
  __syncthreads();
  double mx = -INFINITY;
  for (int m = threadIdx.x; m < G; m += blockDim.x) mx = fmax(mx, s_lam[m]);
  mx = warp_max_d(mx);
  if (lane == 0) s_d[warp] = mx;
  __syncthreads();
  mx = -INFINITY;
  for (int w = 0; w < nw; ++w) mx = fmax(mx, s_d[w]);
  __syncthreads();
  double e = 0.0;
  for (int m = threadIdx.x; m < G; m += blockDim.x) e += s_lam[m] > -INFINITY ? exp(s_lam[m] - mx) : 0.0;
  e = warp_sum_d(e);
  if (lane == 0) s_d[warp] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < nw; ++w) tot += s_d[w];
    s_lc = mx + log(tot);
    a.logZ[t] += s_lc;
  }
  __syncthreads();
  const double lc = s_lc;
  for (int m = threadIdx.x; m < G; m += blockDim.x) {
    const double lam = s_lam[m];
    const long long gm = P.group_off + m;
    a.lam_hist[(long long)a.k * a.G_total + gm] = lam;
    a.lbar_hist[(long long)a.k * a.G_total + gm] = lam - lc;
    if (a.last) a.dlam[gm] = (double)a.seed[t] * exp(lam - lc);
  }
}

// ------------------------------------------------------------------ adjoint
// Log-likelihood (Sec. V model) and its partial derivatives for the
// adjoint: d[0..4] = dl/dx, dl/dy, dl/dI, dl/dsigma_psf, dl/db.  One pass
// over the patch with separable row sums: per row v with r = y - I gx gy,
// R0 = sum r gx, R1 = sum r gx a, R2 = sum r gx a^2 (a the column offset), so
// that sum r gx (u - x) = R1 + du0 R0 and sum r gx (u - x)^2 = R2 + 2 du0 R1
// + du0^2 R0 with du0 = cx - R - x.  Pixels outside the frame count as
// background, so only inside pixels depend on b.
template <int R>
__device__ __forceinline__ float loglik_grad(const float* __restrict__ yp, int pitch, int H, int W, float x, float y,
                                             float I, const TrackParams& P, float (&d)[5]) {
  constexpr int D = 2 * R + 1;
  constexpr int PAD = 2 * R + 1;
  const float cxf = floorf(x + 0.5f), cyf = floorf(y + 0.5f);
  const int cx = (int)fminf(fmaxf(cxf, -(float)(R + 1)), (float)(W + R));
  const int cy = (int)fminf(fmaxf(cyf, -(float)(R + 1)), (float)(H + R));
  const float* __restrict__ row = yp + (long long)(cy - R + PAD) * pitch + (cx - R + PAD);
  float gx[D];
  gauss_row<R>(cxf, x, P.c_psf, P.kappa, gx);
  float gy[D];
  gauss_row<R>(cyf, y, P.c_psf, P.kappa, gy);
  // inside-the-frame column / row ranges of the (true) patch
  const float ulo = fmaxf(0.0f, (float)R - cxf), uhi = fminf((float)(2 * R), (float)(W - 1) + (float)R - cxf);
  const float vlo = fmaxf(0.0f, (float)R - cyf), vhi = fminf((float)(2 * R), (float)(H - 1) + (float)R - cyf);
  float ss = 0.0f, SI = 0.0f, S1 = 0.0f, Sy = 0.0f, Ss = 0.0f, Sb = 0.0f, Y2 = 0.0f, Y1 = 0.0f;
  const float du0 = cxf - (float)R - x;
  // patches wholly inside the frame (almost all) sum the b-derivative's
  // residuals without per-pixel masks
  const bool inside = ulo == 0.0f && uhi == (float)(2 * R) && vlo == 0.0f && vhi == (float)(2 * R);
  auto rows = [&](auto inside_tag) {
    constexpr bool IN = decltype(inside_tag)::value;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const float* __restrict__ rp = row + (long long)b * pitch;
      const float Igy = I * gy[b];
      float R0 = 0.0f, R1 = 0.0f, R2 = 0.0f, Rb = 0.0f;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const float yv = __ldg(rp + a);  // y = z - b, 0 outside the frame
        const float r = fmaf(-gx[a], Igy, yv);
        ss = fmaf(r, r, ss);
        Y2 = fmaf(yv, yv, Y2);
        Y1 += yv;
        const float t = r * gx[a];
        R0 += t;
        R1 = fmaf(t, (float)a, R1);
        R2 = fmaf(t, (float)(a * a), R2);
        if constexpr (IN)
          Rb += r;
        else
          Rb += ((float)a >= ulo && (float)a <= uhi) ? r : 0.0f;
      }
      const float dv = (cyf - (float)R + (float)b) - y;
      const float sx1 = R1 + du0 * R0;
      const float sx2 = R2 + 2.0f * du0 * R1 + du0 * du0 * R0;
      SI = fmaf(gy[b], R0, SI);
      S1 = fmaf(gy[b], sx1, S1);
      Sy = fmaf(gy[b] * dv, R0, Sy);
      Ss = fmaf(gy[b], fmaf(dv * dv, R0, sx2), Ss);
      if (IN || ((float)b >= vlo && (float)b <= vhi)) Sb += Rb;
    }
  };
  if (inside)
    rows(std::true_type{});
  else
    rows(std::false_type{});
  const float iso2 = 2.0f * P.inv2so2;  // 1 / sigma_obs^2
  const float s2 = P.spsf * P.spsf;
  d[0] = I * S1 / s2 * iso2;
  d[1] = I * Sy / s2 * iso2;
  d[2] = SI * iso2;
  d[3] = I * Ss / (s2 * P.spsf) * iso2;
  d[4] = Sb * iso2;
  if (P.obs_model == 1) {
    // frame likelihood ratio: + sum y^2 / (2 sigma_obs^2), whose only
    // parameter is b (dy/db = -1 inside the frame, y = 0 outside)
    d[4] -= Y1 * iso2;
    return -(ss - Y2) * P.inv2so2;
  }
  return -ss * P.inv2so2;
}

template <int R>
__global__ void __launch_bounds__(256, 3) k_adjoint(AdjointArgs a) {
  const int k = a.k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double s_g[8][5];
  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int4 td = a.tiles[tile];
    const TrackParams& P = a.trk[td.x];
    const int g = td.y, Np = P.Np;
    const long long Nt = (long long)P.G * Np;
    const int hslot = k % a.history;
    const float log_G = logf((float)P.G), log_Np = logf((float)Np);
    const bool A_enters = (P.init_kind == INIT_POINT) || (P.init_kind == INIT_SHARING && g == 0);
    float gacc[5] = {0, 0, 0, 0, 0};
    for (int jj = threadIdx.x; jj < td.w; jj += blockDim.x) {
      const int j = td.z + jj;
      const long long il = (long long)g * Np + j, i = P.part_off + il;
      const float4 s = a.pv[i];
      const float I = a.In[i];
      long long par = il;
      int o = g;
      if (k >= 1) {
        par = a.parent[P.parent_off + (long long)hslot * Nt + il];
        o = (int)fastdiv((uint32_t)par, P.m_Np);  // origin group (par < 2^31)
      }
      float dl[5];
      const float l = loglik_grad<R>(a.ypad + P.ypad_off, P.pitch, P.H, P.W, s.x, s.y, I, P, dl);
      const float lb = k >= 1 ? (float)a.lbar_prev[P.group_off + o] : -log_G;
      const float lw = lb - log_Np + l;
      const float lam = (float)a.lam_k[P.group_off + g];
      const float wbar = (lw == lw && lw - lam > -87.0f) ? __expf(lw - lam) : 0.0f;
      const float dlw = (float)a.dlam_k[P.group_off + g] * wbar;
      if (k >= 1) {
        // dL_{k-1} of the origin group: the tile's slots originate in g or in
        // its ring predecessor, so a warp adds two sums instead of 32 terms
        // (slots of any third origin add theirs directly)
        const unsigned full = __activemask();
        const int other = __reduce_max_sync(full, o != g ? o : -1);
        const bool third = o != g && o != other;
        const float own = warp_sum_active(full, (o == g) ? dlw : 0.0f);
        const float pre = warp_sum_active(full, (o != g && !third) ? dlw : 0.0f);
        const int leader = __ffs(full) - 1;
        if (lane == leader) {
          if (own != 0.0f) atomicAdd(&a.D[P.group_off + g], (double)own);
          if (other >= 0 && pre != 0.0f) atomicAdd(&a.D[P.group_off + other], (double)pre);
        }
        if (third && dlw != 0.0f) atomicAdd(&a.D[P.group_off + o], (double)dlw);
      }
      // adjoint of the state: the likelihood term plus the children's
      float4 c = a.Cc_pv[i];
      float cI = a.Cc_I[i];
      a.Cc_pv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      a.Cc_I[i] = 0.0f;
      c.x = fmaf(dlw, dl[0], c.x);
      c.y = fmaf(dlw, dl[1], c.y);
      cI = fmaf(dlw, dl[2], cI);
      gacc[0] = fmaf(dlw, dl[3], gacc[0]);  // sigma_psf
      gacc[2] = fmaf(dlw, dl[4], gacc[2]);  // background
      if (k >= 1) {
        uint4 w0 = make_uint4(j, g, k, P.tag | (ST_PROP << 4) | 0u);
        uint4 w1 = make_uint4(j, g, k, P.tag | (ST_PROP << 4) | 1u);
        philox2(P.key0, P.key1, w0, w1);
        float e0, e1, e2, e3, e4, e5;
        box_muller_fast(w0.x, w0.y, e0, e1);
        box_muller_fast(w0.z, w0.w, e2, e3);
        box_muller_fast(w1.x, w1.y, e4, e5);
        gacc[3] = fmaf(c.x, e0, fmaf(c.y, e1, gacc[3]));  // sigma_pos
        gacc[4] = fmaf(c.z, e2, fmaf(c.w, e3, gacc[4]));  // sigma_v
        // NCV Jacobian transposed onto the parent: x <- x, vx <- x + vx, ...
        // Resampled children of one parent sit in neighbouring slots: lanes
        // sharing a parent add their terms first, one lane stores the sum.
        const long long pi = P.part_off + par;
        float t[5] = {c.x, c.y, c.x + c.z, c.y + c.w, cI};
        const unsigned peers = __match_any_sync(__activemask(), (unsigned long long)pi);
        if (peers != (1u << lane)) {
#pragma unroll
          for (int q = 0; q < 5; ++q) t[q] = warp_sum_active(peers, t[q]);
        }
        if (lane == __ffs(peers) - 1) {
          atomicAdd(&a.Cp_pv[pi].x, t[0]);
          atomicAdd(&a.Cp_pv[pi].y, t[1]);
          atomicAdd(&a.Cp_pv[pi].z, t[2]);
          atomicAdd(&a.Cp_pv[pi].w, t[3]);
          atomicAdd(&a.Cp_I[pi], t[4]);
        }
      } else if (A_enters) {
        gacc[1] += cI;  // the initial intensity is A
      }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const float v = warp_sum(gacc[q]);
      if (lane == 0) s_g[warp][q] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_g[w][threadIdx.x];
      if (v != 0.0) atomicAdd(&a.grad[td.x * 5 + threadIdx.x], v);
    }
    __syncthreads();
  }
}

// dL_{k-1,m} = sum of the origin-m log-weight adjoints of step k; reset D.
__global__ void k_adjoint_groups(double* __restrict__ dlam, double* __restrict__ D, int G_total) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < G_total; m += gridDim.x * blockDim.x) {
    dlam[m] = D[m];
    D[m] = 0.0;
  }
}

__global__ void k_grad_out(const double* __restrict__ g, const double* __restrict__ lz, float* __restrict__ out,
                           double* __restrict__ lz_out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * 5; i += gridDim.x * blockDim.x) {
    out[i] = (float)g[i];
    if (lz_out && i % 5 == 0) lz_out[i / 5] = lz[i / 5];
  }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_replay(const ReplayArgs& a, int R, int grid, cudaStream_t s) {
  switch (R) {
    case 1: k_replay<1><<<grid, 256, 0, s>>>(a); break;
    case 2: k_replay<2><<<grid, 256, 0, s>>>(a); break;
    case 3: k_replay<3><<<grid, 256, 0, s>>>(a); break;
    case 4: k_replay<4><<<grid, 256, 0, s>>>(a); break;
    case 5: k_replay<5><<<grid, 256, 0, s>>>(a); break;
    case 6: k_replay<6><<<grid, 256, 0, s>>>(a); break;
    case 7: k_replay<7><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_replay_groups(const ReplayGroupArgs& a, int n_tracks, int max_G, cudaStream_t s) {
  (void)max_G;
  k_replay_groups<<<n_tracks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjointArgs& a, int R, int grid, cudaStream_t s) {
  switch (R) {
    case 1: k_adjoint<1><<<grid, 256, 0, s>>>(a); break;
    case 2: k_adjoint<2><<<grid, 256, 0, s>>>(a); break;
    case 3: k_adjoint<3><<<grid, 256, 0, s>>>(a); break;
    case 4: k_adjoint<4><<<grid, 256, 0, s>>>(a); break;
    case 5: k_adjoint<5><<<grid, 256, 0, s>>>(a); break;
    case 6: k_adjoint<6><<<grid, 256, 0, s>>>(a); break;
    case 7: k_adjoint<7><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Caller-supplied ancestry for the replay (pf_set_replay): for steps k = 1 ..
// T-1 (blockIdx.y + 1), parents[k * n_total + part_off + il] (track-local
// slot of X_{k-1} that slot il of step k was propagated from) into the
// ancestry record the replay reads.  An index outside the track is counted
// in *bad and recorded as the slot itself, so that no later kernel reads
// outside the track.
__global__ void k_set_replay(const TrackParams* __restrict__ trk, const int4* __restrict__ tiles, int n_tiles,
                             const uint32_t* __restrict__ parents, long long n_total, uint32_t* __restrict__ parent,
                             int history, int* __restrict__ bad) {
  const int k = (int)blockIdx.y + 1;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int4 td = tiles[tile];
    const TrackParams& P = trk[td.x];
    if (!P.record) continue;
    const long long Nt = (long long)P.G * P.Np;
    for (int jj = threadIdx.x; jj < td.w; jj += blockDim.x) {
      const long long il = (long long)td.y * P.Np + td.z + jj;
      uint32_t v = parents[(long long)k * n_total + P.part_off + il];
      if ((long long)v >= Nt) {
        atomicAdd(bad, 1);
        v = (uint32_t)il;
      }
      parent[P.parent_off + (long long)(k % history) * Nt + il] = v;
    }
  }
}

cudaError_t launch_set_replay(const TrackParams* trk, const int4* tiles, int n_tiles, const uint32_t* parents,
                              long long n_total, uint32_t* parent, int history, int T, int* bad, int grid,
                              cudaStream_t s) {
  if (T < 2) return cudaSuccess;
  k_set_replay<<<dim3(grid, T - 1), 256, 0, s>>>(trk, tiles, n_tiles, parents, n_total, parent, history, bad);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_groups(double* dlam, double* D, int G_total, cudaStream_t s) {
  k_adjoint_groups<<<(G_total + 255) / 256, 256, 0, s>>>(dlam, D, G_total);
  return cudaGetLastError();
}

cudaError_t launch_grad_out(const double* g, const double* lz, float* out, double* lz_out, int n, cudaStream_t s) {
  k_grad_out<<<(n * 5 + 255) / 256, 256, 0, s>>>(g, lz, out, lz_out, n);
  return cudaGetLastError();
}

}  // namespace pf
