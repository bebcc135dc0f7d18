// pf_math.cuh -- device arithmetic shared by the step kernels and the
// adjoint kernels of libpfarna: warp / block reductions, the Gaussian-PSF
// patch sums of the likelihood (Sec. V appearance model), Box-Muller
// normals, Philox blocks in lockstep.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "pf_device.cuh"

namespace pf {

// Programmatic dependent launch: wait for the previous kernel in the stream
// (its completion and memory), and allow the next kernel to start.  Both
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
// Sum over the lanes of `mask` (every lane of the mask calls it; the
// result reaches all of them).
__device__ __forceinline__ float warp_sum_active(unsigned mask, float v) {
  if (mask == 0xffffffffu) return warp_sum(v);
  float s = 0.0f;
  for (unsigned m = mask; m; m &= m - 1) s += __shfl_sync(mask, v, __ffs(m) - 1);
  return s;
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


// ===================================================================== likelihood / dynamics helpers
// Gaussian profile values 2^(-c (u - x)^2) on the D = 2R+1 patch columns
// u = cf - R .. cf + R, by a ratio recurrence from the centre column
// outwards: g(u+1) = g(u) r(u), r(u+1) = r(u) 2^(-2c).  Three MUFU ex2 per
// axis instead of D; relative error <= 2R FP32 roundings.
template <int R>
__device__ __forceinline__ void gauss_row(float cf, float x, float c, float kappa, float (&g)[2 * R + 1]) {
  const float d = cf - x;                        // centre offset, |d| <= 1/2
  g[R] = ex2(-c * d * d);
  float up = ex2(-c * fmaf(2.0f, d, 1.0f));      // g(R+1) / g(R)
  float dn = ex2(c * fmaf(2.0f, d, -1.0f));      // g(R-1) / g(R)
#pragma unroll
  for (int a = 1; a <= R; ++a) {
    g[R + a] = g[R + a - 1] * up;
    g[R - a] = g[R - a + 1] * dn;
    up *= kappa;
    dn *= kappa;
  }
}

// gauss_row scaled by `scale` (the spot intensity I): the centre value is
// scale 2^(-c d^2) and the recurrence carries the factor.  The two sides of
// the recurrence advance together in packed FP32 pairs (one FMUL2 per pair
// of products, each lane rounded as its scalar product would be).
template <int R>
__device__ __forceinline__ void gauss_row_scaled(float cf, float x, float c, float kappa, float scale,
                                                 float (&g)[2 * R + 1]) {
  const float d = cf - x;
  g[R] = scale * ex2(-c * d * d);
  float2 ud = make_float2(ex2(-c * fmaf(2.0f, d, 1.0f)), ex2(c * fmaf(2.0f, d, -1.0f)));  // (up, dn)
  const float2 kk = make_float2(kappa, kappa);
  float2 gv = make_float2(g[R], g[R]);
#pragma unroll
  for (int a = 1; a <= R; ++a) {
    gv = __fmul2_rn(gv, ud);
    g[R + a] = gv.x;
    g[R - a] = gv.y;
    ud = __fmul2_rn(ud, kk);
  }
}

// The likelihood's patch sum (Alg. 1 step U, Sec. V appearance model).
// pix(b, a) is the pixel y = z - b of patch row b (0 .. 2R), column a (0
// outside the frame); gxI[a] = I gx(a).  Rows are visited centre-out so that
// gy follows the same ratio recurrence as gauss_row with four live
// registers (dy = cyf - y).
//  FRAME = false (patch residual): sum (y - I gx gy)^2; even and odd
//    columns accumulate on two FMA chains, summed at the end.
//  FRAME = true (frame likelihood ratio): sum [(y - I gx gy)^2 - y^2]
//    = sum m (m - 2y) with m = I gx gy, per pixel (its rounding stays
//    relative to the terms, which stay small where the ratio is small).
// Every pixel source below reads the same pixels in the same order, so all
// give bit-identical sums.
template <int R, bool FRAME, class Pix>
__device__ __forceinline__ float patch_sum(Pix pix, const float (&gxI)[2 * R + 1], float dy, float c, float kappa) {
  float ae = 0.0f, ao = 0.0f;  // even and odd columns
  auto row = [&](int b, float gy) {
    if constexpr (FRAME) {
#pragma unroll
      for (int a = 0; a < 2 * R + 1; ++a) {
        const float m = gxI[a] * gy;
        const float t = fmaf(-2.0f, pix(b, a), m);
        if (a & 1)
          ao = fmaf(m, t, ao);
        else
          ae = fmaf(m, t, ae);
      }
    } else {
#pragma unroll
      for (int a = 0; a < 2 * R + 1; ++a) {
        const float r = fmaf(-gxI[a], gy, pix(b, a));
        if (a & 1)
          ao = fmaf(r, r, ao);
        else
          ae = fmaf(r, r, ae);
      }
    }
  };
  const float g = ex2(-c * dy * dy);
  float up = ex2(-c * fmaf(2.0f, dy, 1.0f));
  float dn = ex2(c * fmaf(2.0f, dy, -1.0f));
  row(R, g);
  float gu = g, gd = g;
#pragma unroll
  for (int a = 1; a <= R; ++a) {
    gu *= up;
    gd *= dn;
    up *= kappa;
    dn *= kappa;
    row(R + a, gu);
    row(R - a, gd);
  }
  return ae + ao;
}

// Rows of shared memory (pitch ROI_W) or of the padded frame in global
// memory (read through L1).
template <int R, bool FRAME, bool SMEM>
__device__ __forceinline__ float patch_ss(const float* __restrict__ base, int pitch, const float (&gxI)[2 * R + 1],
                                          float dy, float c, float kappa) {
  if constexpr (SMEM)
    return patch_sum<R, FRAME>([&](int b, int a) { return base[b * ROI_W + a]; }, gxI, dy, c, kappa);
  else
    return patch_sum<R, FRAME>([&](int b, int a) { return __ldg(base + (long long)b * pitch + a); }, gxI, dy, c,
                               kappa);
}

// Shared-memory rows read as float pairs: `base` is 8-byte aligned and row
// b's pixels are base[b ROI_W + 0 .. 2R] (the pair loads also fetch
// base[.. + 2R + 1], unused).  Columns 2p and 2p + 1 are processed as one
// packed FP32 pair (FFMA2 / FMUL2): lane x is the even column, lane y the
// odd one, so the even and odd accumulators of patch_sum become the two
// lanes of one pair and every lane rounds as the scalar form does; the
// last (even) column goes through the scalar path.  The result is therefore
// bit-identical to patch_sum over the same pixels, in about half the
// instructions.
template <int R, bool FRAME>
__device__ __forceinline__ float patch_ss_pairs(const float* __restrict__ base, const float (&gxI)[2 * R + 1],
                                                float dy, float c, float kappa) {
  float2 gp[R];  // (gx(2p), gx(2p+1)), negated for the residual form
#pragma unroll
  for (int p = 0; p < R; ++p)
    gp[p] = FRAME ? make_float2(gxI[2 * p], gxI[2 * p + 1]) : make_float2(-gxI[2 * p], -gxI[2 * p + 1]);
  float2 acc = make_float2(0.0f, 0.0f);  // (even columns, odd columns)
  auto row = [&](int b, float gy) {
    const float2* __restrict__ r2 = reinterpret_cast<const float2*>(base + b * ROI_W);
    const float2 gy2 = make_float2(gy, gy);
#pragma unroll
    for (int p = 0; p < R; ++p) {
      const float2 y = r2[p];
      if constexpr (FRAME) {
        const float2 m = __fmul2_rn(gp[p], gy2);
        const float2 t = __ffma2_rn(make_float2(-2.0f, -2.0f), y, m);
        acc = __ffma2_rn(m, t, acc);
      } else {
        const float2 r = __ffma2_rn(gp[p], gy2, y);
        acc = __ffma2_rn(r, r, acc);
      }
    }
    const float y = r2[R].x;  // column 2R
    if constexpr (FRAME) {
      const float m = gxI[2 * R] * gy;
      acc.x = fmaf(m, fmaf(-2.0f, y, m), acc.x);
    } else {
      const float r = fmaf(-gxI[2 * R], gy, y);
      acc.x = fmaf(r, r, acc.x);
    }
  };
  const float g = ex2(-c * dy * dy);
  float2 ud = make_float2(ex2(-c * fmaf(2.0f, dy, 1.0f)), ex2(c * fmaf(2.0f, dy, -1.0f)));  // (up, dn)
  const float2 kk = make_float2(kappa, kappa);
  row(R, g);
  float2 gv = make_float2(g, g);  // (rows below the centre, rows above)
#pragma unroll
  for (int a = 1; a <= R; ++a) {
    gv = __fmul2_rn(gv, ud);
    ud = __fmul2_rn(ud, kk);
    row(R + a, gv.x);
    row(R - a, gv.y);
  }
  return acc.x + acc.y;
}

// The caller's frame z (W x H, pitch W) instead of the padded frame: pixel
// values z - b inside the frame, 0 outside; (x0, y0) is the patch's corner
// in frame coordinates.
template <int R, bool FRAME>
__device__ __forceinline__ float patch_ss_raw(const float* __restrict__ z, int W, int H, float bg, int x0, int y0,
                                              const float (&gxI)[2 * R + 1], float dy, float c, float kappa) {
  return patch_sum<R, FRAME>(
      [&](int b, int a) {
        const int yy = y0 + b, xx = x0 + a;
        return ((unsigned)yy < (unsigned)H && (unsigned)xx < (unsigned)W)
                   ? __fsub_rn(__ldg(z + (long long)yy * W + xx), bg)
                   : 0.0f;
      },
      gxI, dy, c, kappa);
}

// Natural log of a uniform u = ((w >> 9) + 1/2) 2^-23: MUFU log2 where its
// absolute error (2^-22 on [1/2, 2]) is small against |ln u|, and the series
// -(t + t^2/2 + t^3/3), t = 1 - u, for the top 2^-10 of the interval.
__device__ __forceinline__ float log_u01(float u) {
  const float t = 1.0f - u;  // exact
  const float series = -t * fmaf(t, fmaf(t, 0.333333343f, 0.5f), 1.0f);
  return t < 9.765625e-4f ? series : __log2f(u) * 0.693147182f;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller pair (see box_muller in pf_device.cuh for the definition).
__device__ __forceinline__ void box_muller_fast(uint32_t wa, uint32_t wb, float& e0, float& e1) {
  const float rho = sqrt_approx(-2.0f * log_u01(u01(wa)));
  float s, c;
  __sincosf(fmaf(u01(wb), 6.28318530717958647f, -3.14159265358979323f), &s, &c);
  e0 = -rho * c;
  e1 = -rho * s;
}

// Two Philox4x32-10 blocks with the round keys given (TrackParams::rk: in
// the kernel's constant bank they are operands, not computed).
__device__ __forceinline__ void philox2_rk(const uint32_t (&rk)[20], uint4& c, uint4& d) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x, p1 = (unsigned long long)0xCD9E8D57u * c.z;
    const unsigned long long q0 = (unsigned long long)0xD2511F53u * d.x, q1 = (unsigned long long)0xCD9E8D57u * d.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                   (uint32_t)p0);
    d = make_uint4((uint32_t)(q1 >> 32) ^ d.y ^ rk[2 * r], (uint32_t)q1, (uint32_t)(q0 >> 32) ^ d.w ^ rk[2 * r + 1],
                   (uint32_t)q0);
  }
}

// Two Philox4x32-10 blocks of the same key in lockstep (shared key schedule).
__device__ __forceinline__ void philox2(uint32_t k0, uint32_t k1, uint4& c, uint4& d) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x, p1 = (unsigned long long)0xCD9E8D57u * c.z;
    const unsigned long long q0 = (unsigned long long)0xD2511F53u * d.x, q1 = (unsigned long long)0xCD9E8D57u * d.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    d = make_uint4((uint32_t)(q1 >> 32) ^ d.y ^ k0, (uint32_t)q1, (uint32_t)(q0 >> 32) ^ d.w ^ k1, (uint32_t)q0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Sum of 8 values over a warp by recursive halving (reduce-scatter): after
// it, lane l holds the total of value ((l >> 2) & 7) (bit-reversed order
// handled by the caller through `slot`).
__device__ __forceinline__ float warp_reduce8(float (&v)[8], int lane, int& slot) {
  float w4[4], w2[2];
  const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = b16 ? v[i] : v[i + 4];
    const float keep = b16 ? v[i + 4] : v[i];
    w4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b8 ? w4[i] : w4[i + 2];
    const float keep = b8 ? w4[i + 2] : w4[i];
    w2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = b4 ? w2[0] : w2[1];
  const float keep = b4 ? w2[1] : w2[0];
  float x = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  slot = (b16 ? 4 : 0) + (b8 ? 2 : 0) + (b4 ? 1 : 0);
  return x;
}

// Order-preserving map of a float to an int (for warp max through redux).
__device__ __forceinline__ int float_key(float f) {
  const int i = __float_as_int(f);
  return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float key_float(int i) { return __int_as_float(i ^ ((i >> 31) & 0x7fffffff)); }

}  // namespace pf
