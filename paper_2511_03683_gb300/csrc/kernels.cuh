// Device kernels of libpb.so (sm_103a).
//
// The hot path is the channel sum of Eq. 2 (arXiv:2511.03683), evaluated as a
// streaming segmented reduction over the state-segmented CSR list: every work item
// is a contiguous piece of one state's row, one warp streams it with 128-bit loads,
// gathers the partner occupations from shared memory, reduces with warp shuffles
// and writes one partial per item; a finaliser adds each row's partials in a fixed
// order.  No global atomics anywhere (the paper's motivation for its target layer,
// Sec. "Optimized GPU algorithm"), and results are deterministic run to run.
//
// Algebra used by the coefficient variants.  With G_a = G(x+w), G_e = G(x-w):
//   term_c = f_s (1-f_p) P_out - (1-f_s) f_p P_in,
//   P_out  = g2 [G_a N + G_e (N+1)]   (rate s -> p),
//   P_in   = g2 [G_a (N+1) + G_e N]   (rate p -> s),   D = P_out - P_in = g2 (G_e - G_a),
// so  I_s = c [ A_s - f_s (R_s - B_s) ],  A_s = sum f_p P_in,  B_s = sum f_p D,
//     R_s = sum P_out,  and  1/tau_s = c (R_s - B_s),  c = 2 pi / (hbar N_q).
// This is Eq. 2 with F_abs, F_em expanded (exact up to rounding order).
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace pb {
namespace dev {

struct Item {
  long long start;  // first channel (padded CSR offset; multiple of 8)
  int len;          // channels (multiple of 8)
  int row;          // window state
};

constexpr int kBlock = 256;  // threads per CTA of the streaming kernels
constexpr int kEntryPad = 8;  // rows of every stream are padded to a multiple of this many entries

// Per-item partial sums (up to three accumulators plus one spare), 32-byte aligned.
struct alignas(32) Part4 {
  double x, y, z, w;
};

__device__ __forceinline__ Part4 make_part4(double x, double y, double z, double w) {
  Part4 p;
  p.x = x;
  p.y = y;
  p.z = z;
  p.w = w;
  return p;
}

// ------------------------------------------------------------ float-float helpers
// A float-float value is hi + lo with |lo| <= ulp(hi)/2: a 48-bit significand with the
// FP32 exponent range.  Error-free transformations (Dekker 1971, Knuth TwoSum) use
// explicitly rounded intrinsics so the compiler never contracts them.

__device__ __forceinline__ float2 ff_split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

__device__ __forceinline__ double ff_to_double(float h, float l) { return (double)h + (double)l; }

// (h, l) += x * (ah, al)
__device__ __forceinline__ void ff_mac(float &h, float &l, float2 x, float ah, float al) {
  const float p = __fmul_rn(x.x, ah);
  float e = __fmaf_rn(x.x, ah, -p);
  e = __fmaf_rn(x.x, al, e);
  e = __fmaf_rn(x.y, ah, e);
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  err = __fadd_rn(err, __fadd_rn(l, e));
  h = __fadd_rn(s, err);
  l = __fsub_rn(err, __fsub_rn(h, s));
}

__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  err = __fadd_rn(err, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, err);
  return make_float2(h, __fsub_rn(err, __fsub_rn(h, s)));
}

__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// Sum over the warp of a float-float value with a fixed xor shuffle tree (FP32 only), then
// one conversion: lane 0's result is reproducible run to run.
__device__ __forceinline__ float2 warp_reduce_ff(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = ff_add(v, make_float2(__shfl_xor_sync(0xFFFFFFFFu, v.x, o), __shfl_xor_sync(0xFFFFFFFFu, v.y, o)));
  return v;
}

__device__ __forceinline__ double warp_sum_ff(float2 v) {
  v = warp_reduce_ff(v);
  return ff_to_double(v.x, v.y);
}

// Exact FP32 -> FP64 widening with integer operations, from the IEEE 754 binary32 and binary64
// layouts: the exponent is rebiased by 1023 - 127 and the significand moves up 29 bits.  Zero
// and subnormal inputs (below 2^-126 in magnitude) give a signed zero; Inf and NaN stay Inf and
// NaN.  Keeps the conversions of float-float results off the FP64 pipe.
__device__ __forceinline__ double widen_f32(float x) {
  const unsigned b = __float_as_uint(x), m = b & 0x7FFFFFFFu, e = m >> 23;
  unsigned hi = (m >> 3) + 0x38000000u, lo = b << 29;
  if (e == 0u) hi = lo = 0u;
  if (e == 0xFFu) hi |= 0x7FF00000u;
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// reduce-scatter of NV float-float values over the 2 * TOP lanes that differ in lane bits
// log2 TOP .. 0: at the end v[0] holds, on every lane, the total of value index idx(lane) = those
// bits of the lane, most significant first (the first log2 NV of them).  Full float-float
// additions: the low words of lazily added partials of many lanes would grow to many ulps of the
// high word, and their FP32 rounding with them.
template <int NV, int TOP>
__device__ __forceinline__ void ff_reduce_scatter(float2 (&v)[NV], int lane) {
  int n = NV;
#pragma unroll
  for (int mask = TOP; mask > 0; mask >>= 1) {
    if (n > 1) {
      const bool up = lane & mask;
      const int h = n >> 1;
#pragma unroll
      for (int k = 0; k < NV / 2; ++k) {
        if (k < h) {
          const float2 send = up ? v[k] : v[k + h], keep = up ? v[k + h] : v[k];
          const float2 recv = make_float2(__shfl_xor_sync(0xFFFFFFFFu, send.x, mask),
                                          __shfl_xor_sync(0xFFFFFFFFu, send.y, mask));
          v[k] = ff_add(keep, recv);
        }
      }
      n = h;
    } else {
      v[0] = ff_add(v[0], make_float2(__shfl_xor_sync(0xFFFFFFFFu, v[0].x, mask),
                                      __shfl_xor_sync(0xFFFFFFFFu, v[0].y, mask)));
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double gauss(double x, double inv2s2, double norm) { return norm * exp(-x * x * inv2s2); }

__device__ __forceinline__ int q_of(short4 ks, short4 kp, int N1, int N2, int N3) {
  int d1 = kp.x - ks.x, d2 = kp.y - ks.y, d3 = kp.z - ks.z;
  d1 += d1 < 0 ? N1 : 0;
  d2 += d2 < 0 ? N2 : 0;
  d3 += d3 < 0 ? N3 : 0;
  return (d1 * N2 + d2) * N3 + d3;
}

// ------------------------------------------------------------ setup kernels

// (hbar w, N) per (q, nu); N = 1/(exp(w/kT)-1) for w > 0, else 0 (such channels are not stored)
__global__ void k_table(const double *__restrict__ omega, long long n, double kT, double2 *__restrict__ tab) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double w = omega[i];
    tab[i] = make_double2(w, w > 0.0 ? 1.0 / expm1(w / kT) : 0.0);
  }
}

__global__ void k_to_ff(const double *__restrict__ x, long long n, float2 *__restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = ff_split(x[i]);
}

// the same into a padded state space: out[pmap[i]] (the padding keeps its zeros)
__global__ void k_to_ff_map(const double *__restrict__ x, int n, const int *__restrict__ pmap,
                            float2 *__restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[pmap[i]] = ff_split(x[i]);
}

struct ChanGeom {
  const uint32_t *col;   // packed partner | nu << 24
  const double *g2;      // |g|^2 per channel (0 on padding)
  const double *eps;     // [ns]
  const short4 *kc;      // [ns] grid coordinates
  const double2 *tab;    // [nq][nmodes] (w, N)
  int N1, N2, N3, nmodes;
  double inv2s2, norm;   // 1/(2 sigma^2), 1/(sqrt(2 pi) sigma)
};

__device__ __forceinline__ void channel_deltas(const ChanGeom &g, int r, uint32_t cw, double &g2, double &Ga,
                                               double &Ge, double &N, int &p, long long c) {
  p = (int)(cw & 0xFFFFFFu);
  const int nu = (int)(cw >> 24);
  const int iq = q_of(g.kc[r], g.kc[p], g.N1, g.N2, g.N3);
  const double2 wN = g.tab[(long long)iq * g.nmodes + nu];
  const double x = g.eps[r] - g.eps[p];
  g2 = g.g2[c];
  Ga = gauss(x + wN.x, g.inv2s2, g.norm);
  Ge = gauss(x - wN.x, g.inv2s2, g.norm);
  N = wN.y;
}

// Per-channel rate coefficients (P_in, D) in FP64, stored as float-float (FF=true) or
// double; part[item].x = sum over the item of P_out (for R_s).  KFORM stores them without
// the factor |g|^2 (P_in / g2 = G_a (N+1) + G_e N, D / g2 = G_e - G_a): the branch-merged
// devices keep that form per channel, for the branch sums (which multiply g2 back in) and
// for the |g|^2 gradient (whose bracket is exactly that form).
template <bool FF, bool KFORM = false>
__global__ void __launch_bounds__(kBlock) k_coef(const Item *__restrict__ items, int nitems, ChanGeom g,
                                                 void *__restrict__ coefA, void *__restrict__ coefB,
                                                 Part4 *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    double acc = 0.0;
    for (int j = lane; j < I.len; j += 32) {
      const long long c = I.start + j;
      double g2, Ga, Ge, N;
      int p;
      channel_deltas(g, I.row, g.col[c], g2, Ga, Ge, N, p, c);
      const double kin = Ga * (N + 1.0) + Ge * N, kd = Ge - Ga;
      const double pin = KFORM ? kin : g2 * kin;
      const double dd = KFORM ? kd : g2 * kd;
      acc += g2 * (Ga * N + Ge * (N + 1.0));
      if (FF) {
        ((float2 *)coefA)[c] = ff_split(pin);
        ((float2 *)coefB)[c] = ff_split(dd);
      } else {
        ((double *)coefA)[c] = pin;
        ((double *)coefB)[c] = dd;
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) part[it] = make_part4(acc, 0.0, 0.0, 0.0);
  }
}

// Branch-merged coefficients.  For fixed eps, omega, sigma and T every branch nu of a state
// pair (s, p) enters Eq. 2 through the same f_s and f_p, so the coefficient form only needs
// the sums over nu:  P_in(s,p) = sum_nu P_in(s,p,nu),  D(s,p) = sum_nu D(s,p,nu).  Entry k
// sums the cnt[k] consecutive channels from cstart[k] in FP64 (ascending nu), each times
// w[channel] when w is given (the g2 of coefficients stored without it), multiplies by
// scale and stores the result in the sweep's format; padding entries (cnt 0) become zero.
template <bool FF>
__global__ void k_pair_coef(const long long *__restrict__ cstart, const uint8_t *__restrict__ cnt, long long n,
                            const void *__restrict__ cA, const void *__restrict__ cB, void *__restrict__ pA,
                            void *__restrict__ pB, double scale, const double *__restrict__ w) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long s = cstart[k];
    const int m = cnt[k];
    double a = 0.0, b = 0.0;
    for (int i = 0; i < m; ++i) {
      double x, y;
      if (FF) {
        const float2 xf = ((const float2 *)cA)[s + i], yf = ((const float2 *)cB)[s + i];
        x = ff_to_double(xf.x, xf.y);
        y = ff_to_double(yf.x, yf.y);
      } else {
        x = ((const double *)cA)[s + i];
        y = ((const double *)cB)[s + i];
      }
      if (w) {
        x *= w[s + i];
        y *= w[s + i];
      }
      a += x;
      b += y;
    }
    a *= scale;
    b *= scale;
    if (FF) {
      ((float2 *)pA)[k] = ff_split(a);
      ((float2 *)pB)[k] = ff_split(b);
    } else {
      ((double *)pA)[k] = a;
      ((double *)pB)[k] = b;
    }
  }
}

// dst[i] = scale * src[i]
__global__ void k_scale_copy(const double *__restrict__ src, int n, double scale, double *__restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = scale * src[i];
}

// Transport weights from the coefficient arrays: W = c (P_in + (1 - f0_p) D), which equals
// c g2 [G_a (N + f0_p) + G_e (N + 1 - f0_p)] summed over the entry's channels; stored
// float-float; part[item].x = sum of W over the item.
template <bool FF, typename IDX>
__global__ void __launch_bounds__(kBlock) k_weights_coef(const Item *__restrict__ items, int nitems,
                                                         const void *__restrict__ cA, const void *__restrict__ cB,
                                                         const IDX *__restrict__ colp, const double *__restrict__ f0,
                                                         double cpref, float2 *__restrict__ wt,
                                                         Part4 *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    double acc = 0.0;
    for (int j = lane; j < I.len; j += 32) {
      const long long c = I.start + j;
      double a, b;
      if (FF) {
        const float2 x = ((const float2 *)cA)[c], y = ((const float2 *)cB)[c];
        a = ff_to_double(x.x, x.y);
        b = ff_to_double(y.x, y.y);
      } else {
        a = ((const double *)cA)[c];
        b = ((const double *)cB)[c];
      }
      const unsigned p = (unsigned)colp[c] & 0xFFFFFFu;
      const double W = cpref * (a + (1.0 - f0[p]) * b);
      wt[c] = ff_split(W);
      acc += W;
    }
    acc = warp_sum(acc);
    if (lane == 0) part[it] = make_part4(acc, 0.0, 0.0, 0.0);
  }
}

// Transport weights W_c = c g2 [G_a (N + f0_p) + G_e (N + 1 - f0_p)] stored float-float;
// part[item].x = sum of W over the item (for 1/tau_s at f0).
__global__ void __launch_bounds__(kBlock) k_weights(const Item *__restrict__ items, int nitems, ChanGeom g,
                                                    const double *__restrict__ f0, double cpref,
                                                    float2 *__restrict__ wt, Part4 *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    double acc = 0.0;
    for (int j = lane; j < I.len; j += 32) {
      const long long c = I.start + j;
      double g2, Ga, Ge, N;
      int p;
      channel_deltas(g, I.row, g.col[c], g2, Ga, Ge, N, p, c);
      const double fp = f0[p];
      const double W = cpref * g2 * (Ga * (N + fp) + Ge * (N + 1.0 - fp));
      wt[c] = ff_split(W);
      acc += W;
    }
    acc = warp_sum(acc);
    if (lane == 0) part[it] = make_part4(acc, 0.0, 0.0, 0.0);
  }
}

// out[r] = sum of part[i].x over the items of row r, in item order
__global__ void k_rowsum(const int *__restrict__ item_ptr, const Part4 *__restrict__ part, int ns,
                         double *__restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ns) return;
  double s = 0.0;
  for (int i = item_ptr[r]; i < item_ptr[r + 1]; ++i) s += part[i].x;
  out[r] = s;
}

__global__ void k_recip(const double *__restrict__ x, int n, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[i] > 0.0 ? 1.0 / x[i] : 0.0;
}

// Partner indices of the 4-channel group q, from the packed 32-bit words (partner in the
// low 24 bits) or from the compact 16-bit copy kept when nstate <= 65536.
template <typename IDX>
__device__ __forceinline__ uint4 partners4(const IDX *__restrict__ col, long long q);
template <>
__device__ __forceinline__ uint4 partners4<uint32_t>(const uint32_t *__restrict__ col, long long q) {
  const uint4 c = __ldcs((const uint4 *)col + q);
  return make_uint4(c.x & 0xFFFFFFu, c.y & 0xFFFFFFu, c.z & 0xFFFFFFu, c.w & 0xFFFFFFu);
}
template <>
__device__ __forceinline__ uint4 partners4<uint16_t>(const uint16_t *__restrict__ col, long long q) {
  const uint2 c = __ldcs((const uint2 *)col + q);
  return make_uint4(c.x & 0xFFFFu, c.x >> 16, c.y & 0xFFFFu, c.y >> 16);
}

// ------------------------------------------------------------ streaming kernels
enum { MODE_COLL = 0, MODE_RATE = 1, MODE_VJP = 2 };  // MODE_VJP: the dense mixed-precision sweep only

// The four occupations (float-float) of the entries of group q (4 consecutive entries): gathered
// through their partner indices, or, for complete rows (DENSE: the row's entries are its
// partners 0, 1, 2, ... in order), read as two 16-byte words from shared memory at pe, the
// partner of the group's first entry.
template <bool DENSE, typename IDX>
__device__ __forceinline__ void group_f(const float2 *__restrict__ fv, const IDX *__restrict__ colp, long long q,
                                        int pe, float2 &f0, float2 &f1, float2 &f2, float2 &f3) {
  if (DENSE) {
    const float4 x = ((const float4 *)fv)[pe >> 1], y = ((const float4 *)fv)[(pe >> 1) + 1];
    f0 = make_float2(x.x, x.y);
    f1 = make_float2(x.z, x.w);
    f2 = make_float2(y.x, y.y);
    f3 = make_float2(y.z, y.w);
  } else {
    const uint4 c = partners4(colp, q);
    f0 = fv[c.x];
    f1 = fv[c.y];
    f2 = fv[c.z];
    f3 = fv[c.w];
  }
}

// Float-float coefficient stream.  Entry c (a channel, or a state pair of the branch-merged
// sweep): coefA[c] = P_in (hi,lo), coefB[c] = D (hi,lo), colp = partner index.  One warp per
// item, each lane two 4-entry groups per trip.
// part[item] = (A, B) where A = sum f_p P_in, B = sum f_p D (MODE_RATE: only B).
// DENSE (with SMEM only): complete rows, no index stream; srp holds the rows' first entries
// and the shared-memory copy of f is zero-padded to a multiple of kEntryPad states.
template <int MODE, bool SMEM, typename IDX, bool DENSE = false>
__global__ void __launch_bounds__(kBlock) k_stream_ff(const Item *__restrict__ items, int nitems,
                                                      const float4 *__restrict__ A4, const float4 *__restrict__ B4,
                                                      const IDX *__restrict__ colp,
                                                      const float2 *__restrict__ fg, int ns,
                                                      Part4 *__restrict__ part,
                                                      const long long *__restrict__ srp = nullptr) {
  extern __shared__ float2 fsm[];
  if (SMEM) {
    const int nsp = DENSE ? (ns + kEntryPad - 1) / kEntryPad * kEntryPad : ns;
    for (int i = threadIdx.x; i < nsp; i += blockDim.x) fsm[i] = i < ns ? fg[i] : make_float2(0.f, 0.f);
    __syncthreads();
  }
  const float2 *__restrict__ fv = SMEM ? fsm : fg;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long g0 = I.start >> 2;
    const int ng = I.len >> 2;
    const int pb0 = DENSE ? (int)(I.start - srp[I.row]) : 0;  // partner of the item's first entry
    float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
    int g = lane;
    for (; g + 32 < ng; g += 64) {
      const long long q0 = g0 + g, q1 = q0 + 32;
      float2 f0, f1, f2, f3, f4, f5, f6, f7;
      group_f<DENSE>(fv, colp, q0, pb0 + 4 * g, f0, f1, f2, f3);
      group_f<DENSE>(fv, colp, q1, pb0 + 4 * g + 128, f4, f5, f6, f7);
      float4 a00, a01, a10, a11;
      if (MODE == MODE_COLL) {
        a00 = __ldcs(A4 + 2 * q0); a01 = __ldcs(A4 + 2 * q0 + 1);
        a10 = __ldcs(A4 + 2 * q1); a11 = __ldcs(A4 + 2 * q1 + 1);
      }
      const float4 b00 = __ldcs(B4 + 2 * q0), b01 = __ldcs(B4 + 2 * q0 + 1);
      const float4 b10 = __ldcs(B4 + 2 * q1), b11 = __ldcs(B4 + 2 * q1 + 1);
      if (MODE == MODE_COLL) {
        ff_mac(ah, al, f0, a00.x, a00.y); ff_mac(ah, al, f1, a00.z, a00.w);
        ff_mac(ah, al, f2, a01.x, a01.y); ff_mac(ah, al, f3, a01.z, a01.w);
        ff_mac(ah, al, f4, a10.x, a10.y); ff_mac(ah, al, f5, a10.z, a10.w);
        ff_mac(ah, al, f6, a11.x, a11.y); ff_mac(ah, al, f7, a11.z, a11.w);
      }
      ff_mac(bh, bl, f0, b00.x, b00.y); ff_mac(bh, bl, f1, b00.z, b00.w);
      ff_mac(bh, bl, f2, b01.x, b01.y); ff_mac(bh, bl, f3, b01.z, b01.w);
      ff_mac(bh, bl, f4, b10.x, b10.y); ff_mac(bh, bl, f5, b10.z, b10.w);
      ff_mac(bh, bl, f6, b11.x, b11.y); ff_mac(bh, bl, f7, b11.z, b11.w);
    }
    if (g < ng) {
      const long long q0 = g0 + g;
      float2 f0, f1, f2, f3;
      group_f<DENSE>(fv, colp, q0, pb0 + 4 * g, f0, f1, f2, f3);
      if (MODE == MODE_COLL) {
        const float4 a00 = __ldcs(A4 + 2 * q0), a01 = __ldcs(A4 + 2 * q0 + 1);
        ff_mac(ah, al, f0, a00.x, a00.y); ff_mac(ah, al, f1, a00.z, a00.w);
        ff_mac(ah, al, f2, a01.x, a01.y); ff_mac(ah, al, f3, a01.z, a01.w);
      }
      const float4 b00 = __ldcs(B4 + 2 * q0), b01 = __ldcs(B4 + 2 * q0 + 1);
      ff_mac(bh, bl, f0, b00.x, b00.y); ff_mac(bh, bl, f1, b00.z, b00.w);
      ff_mac(bh, bl, f2, b01.x, b01.y); ff_mac(bh, bl, f3, b01.z, b01.w);
    }
    const double A = MODE == MODE_COLL ? warp_sum_ff(make_float2(ah, al)) : 0.0;
    const double B = warp_sum_ff(make_float2(bh, bl));
    if (lane == 0) part[it] = make_part4(A, B, 0.0, 0.0);
  }
}

// ------------------------------------------------------------ TMA bulk-copy form of the sweep
//
// The same float-float collision sweep with the stream staged through shared memory by the
// Tensor Memory Accelerator: one thread issues 1D bulk copies (cp.async.bulk, completion
// counted in bytes on an mbarrier) of each work item's P_in, D and 16-bit index slices into
// a ring of NSTAGE buffers; the whole CTA consumes a buffer, reduces the item, and the buffer
// is refilled.  Each CTA owns a contiguous range of items.  Every wait is bounded in time (a
// try_wait may suspend the thread for a while, so polls are not counted): when it gives up the
// kernel records the failure in *err, waits (bounded) for its own copies and returns; the host
// reads *err.

constexpr int kBulkStages = 4;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait of at most about ns nanoseconds; false when the limit was reached.  The first 1024 polls
// read no clock (the usual waits end there); after them the clock is read every 64 polls, and
// a cap on the polls bounds the loop even without the clock.
constexpr unsigned kWaitPolls = 1u << 24;
__device__ __forceinline__ bool mbar_wait_for(unsigned long long *bar, unsigned parity, unsigned long long ns) {
  for (int i = 0; i < 1024; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned i = 0; i < kWaitPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && globaltimer_ns() - t0 >= ns) return false;
  }
  return false;
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  return mbar_wait_for(bar, parity, kWaitNs);
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Test of the bounded waits: one CTA issues a 1 KB bulk copy (completing on bars[0]), then waits
// on bars[1], which nothing arrives on, for at most `ns` nanoseconds; on the give-up it records
// the failure in *err and waits (bounded) for its own copy, like the sweeps' failure path.
__global__ void k_selftest_wait(const float4 *__restrict__ src, unsigned long long ns, int *__restrict__ err) {
  __shared__ __align__(128) float4 buf[64];
  __shared__ unsigned long long bars[2];
  if (threadIdx.x == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bars, sizeof(buf));
    bulk_g2s(buf, src, sizeof(buf), bars);
    if (!mbar_wait_for(bars + 1, 0, ns)) {
      *err = 4;
      mbar_wait(bars, 0);  // drain the copy in flight
    }
  }
  __syncthreads();
}

// Dynamic shared memory: f table (ns float2), then NSTAGE x [P_in | D | idx] buffers of
// `cap` channels, then NSTAGE mbarriers and the reduction scratch.
__global__ void __launch_bounds__(kBlock) k_stream_ff_bulk(const Item *__restrict__ items, int nitems,
                                                           const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                           const uint16_t *__restrict__ col16,
                                                           const float2 *__restrict__ fg, int ns, int cap,
                                                           Part4 *__restrict__ part, int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char bsm[];
  float2 *fs = (float2 *)bsm;
  const size_t fbytes = ((size_t)ns * sizeof(float2) + 127) / 128 * 128;
  const size_t sbytes = ((size_t)cap * (2 * sizeof(float2) + sizeof(uint16_t)) + 127) / 128 * 128;
  unsigned char *stage0 = bsm + fbytes;
  unsigned long long *bars = (unsigned long long *)(stage0 + kBulkStages * sbytes);
  unsigned long long *fbar = bars + kBulkStages;
  Item *sitem = (Item *)(bars + kBulkStages + 1);   // descriptors of the items in flight
  double *red = (double *)(sitem + kBulkStages);    // [2 * warps]

  const int per = (nitems + gridDim.x - 1) / gridDim.x;
  const int ib = blockIdx.x * per;
  const int ie = min(nitems, ib + per);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;

  if (tid == 0) {
    for (int k = 0; k <= kBulkStages; ++k) mbar_init(bars + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int issued = 0;  // copies issued by thread 0 (stage uses), for the drain on failure
  auto issue = [&](const Item &I, int s) {
    unsigned char *buf = stage0 + (size_t)s * sbytes;
    const unsigned n8 = (unsigned)I.len * sizeof(float2), n2 = (unsigned)I.len * sizeof(uint16_t);
    sitem[s] = I;
    mbar_expect_tx(bars + s, 2 * n8 + n2);
    bulk_g2s(buf, A + I.start, n8, bars + s);
    bulk_g2s(buf + (size_t)cap * sizeof(float2), B + I.start, n8, bars + s);
    bulk_g2s(buf + (size_t)cap * 2 * sizeof(float2), col16 + I.start, n2, bars + s);
  };
  // the f table, rounded up to a 16-byte multiple (the source region is padded to 256 bytes)
  const unsigned fcopy = (unsigned)(((size_t)ns * sizeof(float2) + 15) / 16 * 16);
  if (tid == 0) {
    mbar_expect_tx(fbar, fcopy);
    bulk_g2s(fs, fg, fcopy, fbar);
    for (int it = ib; it < ie && it < ib + kBulkStages; ++it, ++issued) issue(items[it], (it - ib) % kBulkStages);
  }
  // every give-up decision is taken by the whole CTA at once (__syncthreads_and), so no thread
  // is left waiting at a barrier another thread has abandoned
  // thread 0 waits on the mbarrier (acquire); the CTA barrier then orders the staged data for
  // every other thread, so the rest of the CTA sleeps at __syncthreads instead of spinning
  bool ok = __syncthreads_and(tid == 0 ? mbar_wait(fbar, 0) : true);
  for (int it = ib; it < ie && ok; ++it) {
    const int s = (it - ib) % kBulkStages;
    const unsigned parity = (unsigned)(((it - ib) / kBulkStages) & 1);
    // thread 0 fetches the descriptor of the item that will refill this stage while it waits
    Item nextI;
    const bool refill = it + kBulkStages < ie;
    if (tid == 0 && refill) nextI = items[it + kBulkStages];
    if (!__syncthreads_and(tid == 0 ? mbar_wait(bars + s, parity) : true)) {
      ok = false;
      break;
    }
    const int len = sitem[s].len;
    const unsigned char *buf = stage0 + (size_t)s * sbytes;
    const float2 *pa = (const float2 *)buf;
    const float2 *pd = (const float2 *)(buf + (size_t)cap * sizeof(float2));
    const uint16_t *pc = (const uint16_t *)(buf + (size_t)cap * 2 * sizeof(float2));
    float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
    for (int j = tid; j < len; j += blockDim.x) {
      const float2 fp = fs[pc[j]];
      const float2 a = pa[j], b = pd[j];
      ff_mac(ah, al, fp, a.x, a.y);
      ff_mac(bh, bl, fp, b.x, b.y);
    }
    double Ax = warp_sum(ff_to_double(ah, al)), Bx = warp_sum(ff_to_double(bh, bl));
    if (lane == 0) {
      red[2 * wid] = Ax;
      red[2 * wid + 1] = Bx;
    }
    __syncthreads();  // every thread is done with buffer s and has posted its warp sums
    if (tid == 0) {
      if (refill) {
        fence_proxy_async();  // order the generic-proxy reads of buffer s before the async refill
        issue(nextI, s);
        ++issued;
      }
      double a = 0.0, b = 0.0;
      for (int w = 0; w < nw; ++w) {
        a += red[2 * w];
        b += red[2 * w + 1];
      }
      part[it] = make_part4(a, b, 0.0, 0.0);
    }
  }
  if (!ok) {
    *err = 1;
    // drain: wait (bounded) for every copy this CTA issued before leaving
    if (tid == 0) {
      for (int k = 0; k < kBulkStages; ++k) {
        const int uses = issued / kBulkStages + (k < issued % kBulkStages ? 1 : 0);
        if (uses > 0) mbar_wait(bars + k, (unsigned)((uses - 1) & 1));
      }
      mbar_wait(fbar, 0);
    }
  }
}

// Same coefficient stream held as doubles, with native FP64 FMAs (f gathered as double).
template <int MODE, bool SMEM, typename IDX>
__global__ void __launch_bounds__(kBlock) k_stream_f64(const Item *__restrict__ items, int nitems,
                                                       const double2 *__restrict__ A2, const double2 *__restrict__ B2,
                                                       const IDX *__restrict__ colp, const double *__restrict__ fg,
                                                       int ns, Part4 *__restrict__ part) {
  extern __shared__ double fsd[];
  if (SMEM) {
    for (int i = threadIdx.x; i < ns; i += blockDim.x) fsd[i] = fg[i];
    __syncthreads();
  }
  const double *__restrict__ fv = SMEM ? fsd : fg;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long g0 = I.start >> 2;
    const int ng = I.len >> 2;
    double A = 0.0, B = 0.0;
    for (int g = lane; g < ng; g += 32) {
      const long long q = g0 + g;
      const uint4 c = partners4(colp, q);
      const double f0 = fv[c.x], f1 = fv[c.y], f2 = fv[c.z], f3 = fv[c.w];
      if (MODE == MODE_COLL) {
        const double2 a0 = __ldcs(A2 + 2 * q), a1 = __ldcs(A2 + 2 * q + 1);
        A = fma(f0, a0.x, A); A = fma(f1, a0.y, A); A = fma(f2, a1.x, A); A = fma(f3, a1.y, A);
      }
      const double2 b0 = __ldcs(B2 + 2 * q), b1 = __ldcs(B2 + 2 * q + 1);
      B = fma(f0, b0.x, B); B = fma(f1, b0.y, B); B = fma(f2, b1.x, B); B = fma(f3, b1.y, B);
    }
    A = warp_sum(A);
    B = warp_sum(B);
    if (lane == 0) part[it] = make_part4(A, B, 0.0, 0.0);
  }
}

// The literal form: stream |g|^2 and the packed (partner, nu) word, and evaluate the two
// Gaussians, the Bose factor lookup and F_abs / F_em of Eq. 2 in FP64 registers.
// part[item].x = sum of g2 [G_a F_abs + G_e F_em] (MODE_COLL) or of the rate summand.
template <int MODE>
__global__ void __launch_bounds__(kBlock) k_stream_literal(const Item *__restrict__ items, int nitems, ChanGeom g,
                                                           const double *__restrict__ f, Part4 *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const double fs = f[I.row];
    double acc = 0.0;
    for (int j = lane; j < I.len; j += 32) {
      const long long c = I.start + j;
      double g2, Ga, Ge, N;
      int p;
      channel_deltas(g, I.row, __ldcs(g.col + c), g2, Ga, Ge, N, p, c);
      const double fp = f[p];
      if (MODE == MODE_COLL) {
        const double Fabs = fs * (1.0 - fp) * N - (1.0 - fs) * fp * (N + 1.0);
        const double Fem = fs * (1.0 - fp) * (N + 1.0) - (1.0 - fs) * fp * N;
        acc += g2 * (Ga * Fabs + Ge * Fem);
      } else {
        acc += g2 * (Ga * (N + fp) + Ge * (N + 1.0 - fp));
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) part[it] = make_part4(acc, 0.0, 0.0, 0.0);
  }
}

// Transport: stream W (float-float, c folded in) and the partner index; gather F[p][0..2]
// (float-float, [ns][3]) from shared memory (SMEM) or through L1 (__ldg), and accumulate the
// three field directions in one pass, two 4-channel groups per lane per trip.
template <bool SMEM>
__device__ __forceinline__ float2 ldF(const float2 *__restrict__ F, unsigned i) {
  if (SMEM) return F[i];
  return __ldg(F + i);
}

template <bool SMEM>
__device__ __forceinline__ void tr_group(const float2 *__restrict__ Fv, uint4 c, float4 w0, float4 w1, float &xh,
                                         float &xl, float &yh, float &yl, float &zh, float &zl) {
  const unsigned p[4] = {c.x, c.y, c.z, c.w};
  const float wh[4] = {w0.x, w0.z, w1.x, w1.z};
  const float wl[4] = {w0.y, w0.w, w1.y, w1.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned b = 3u * p[k];
    ff_mac(xh, xl, ldF<SMEM>(Fv, b), wh[k], wl[k]);
    ff_mac(yh, yl, ldF<SMEM>(Fv, b + 1), wh[k], wl[k]);
    ff_mac(zh, zl, ldF<SMEM>(Fv, b + 2), wh[k], wl[k]);
  }
}

template <bool SMEM, typename IDX>
__global__ void __launch_bounds__(kBlock) k_stream_tr(const Item *__restrict__ items, int nitems,
                                                      const float4 *__restrict__ W4, const IDX *__restrict__ colp,
                                                      const float2 *__restrict__ Fg, int ns,
                                                      Part4 *__restrict__ part) {
  extern __shared__ float2 Fsm[];
  if (SMEM) {
    for (int i = threadIdx.x; i < 3 * ns; i += blockDim.x) Fsm[i] = Fg[i];
    __syncthreads();
  }
  const float2 *__restrict__ Fv = SMEM ? Fsm : Fg;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long g0 = I.start >> 2;
    const int ng = I.len >> 2;
    float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f, zh = 0.f, zl = 0.f;
    // software pipeline: the next group's weights and indices load while this group computes
    uint4 c = make_uint4(0u, 0u, 0u, 0u);
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0;
    if (lane < ng) {
      c = partners4(colp, g0 + lane);
      w0 = __ldcs(W4 + 2 * (g0 + lane));
      w1 = __ldcs(W4 + 2 * (g0 + lane) + 1);
    }
    for (int g = lane; g < ng; g += 32) {
      uint4 cn = make_uint4(0u, 0u, 0u, 0u);
      float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
      if (g + 32 < ng) {
        const long long qn = g0 + g + 32;
        cn = partners4(colp, qn);
        n0 = __ldcs(W4 + 2 * qn);
        n1 = __ldcs(W4 + 2 * qn + 1);
      }
      tr_group<SMEM>(Fv, c, w0, w1, xh, xl, yh, yl, zh, zl);
      c = cn;
      w0 = n0;
      w1 = n1;
    }
    const double X = warp_sum(ff_to_double(xh, xl));
    const double Y = warp_sum(ff_to_double(yh, yl));
    const double Z = warp_sum(ff_to_double(zh, zl));
    if (lane == 0) part[it] = make_part4(X, Y, Z, 0.0);
  }
}

// (h, l) += x * (ah + al) like ff_mac, but without renormalising (h, l) after every term: h
// takes the exact TwoSum and l collects the rounding errors and cross products in FP32.  Over
// the ~64 terms a lane adds per work item, l stays within about 64 ulp(h), so its own rounding
// costs about 2^-18 ulp(h): the pair is still exact to about 2^-42 relative, at 11 operations
// per term instead of 15.
__device__ __forceinline__ void ff_mac_lazy(float &h, float &l, float2 x, float ah, float al) {
  const float p = __fmul_rn(x.x, ah);
  float e = __fmaf_rn(x.x, ah, -p);
  e = __fmaf_rn(x.x, al, e);
  e = __fmaf_rn(x.y, ah, e);
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  l = __fadd_rn(l, __fadd_rn(err, e));
  h = s;
}

// (h, l) = x * (ah, al): the first term of a lazily accumulated float-float sum (no addition)
__device__ __forceinline__ void ff_prod(float &h, float &l, float2 x, float ah, float al) {
  h = __fmul_rn(x.x, ah);
  float e = __fmaf_rn(x.x, ah, -h);
  e = __fmaf_rn(x.x, al, e);
  l = __fmaf_rn(x.y, ah, e);
}

template <bool LAZY, bool GLOBAL>
__device__ __forceinline__ void tr_mac3(float (&acc)[6], const float2 *Fp, float2 w) {
  const float2 fx = GLOBAL ? __ldg(Fp) : Fp[0], fy = GLOBAL ? __ldg(Fp + 1) : Fp[1], fz = GLOBAL ? __ldg(Fp + 2) : Fp[2];
  if (LAZY) {
    ff_mac_lazy(acc[0], acc[1], fx, w.x, w.y);
    ff_mac_lazy(acc[2], acc[3], fy, w.x, w.y);
    ff_mac_lazy(acc[4], acc[5], fz, w.x, w.y);
  } else {
    ff_mac(acc[0], acc[1], fx, w.x, w.y);
    ff_mac(acc[2], acc[3], fy, w.x, w.y);
    ff_mac(acc[4], acc[5], fz, w.x, w.y);
  }
}

// Transport sweep with consecutive lanes on consecutive channels: a warp's 32 channels share
// about 32/nmodes partners, so each F gather touches few L1 sectors or shared-memory banks;
// weights (8 B) and indices stay fully coalesced across the warp.  Four channels per lane per
// trip.  Shapes: NT = 256 with F gathered through L1 (eight CTAs per SM), or NT = 1024 (one
// CTA per SM) with F staged in shared memory (SMEMF) and the next trip's weights and indices
// loaded into registers before this trip's gathers (RP).  DENSE (with SMEMF only): complete
// rows, the partner of entry j is the entry's position in its row (srp: the rows' first
// entries), no index stream; F in shared memory is zero-padded to a multiple of kEntryPad states.
template <typename IDX, int NT, bool SMEMF, bool RP, bool LAZY, bool DENSE = false>
__global__ void __launch_bounds__(NT, NT == 1024 ? 1 : 8) k_stream_tr_lane(const Item *__restrict__ items, int nitems,
                                                          const float2 *__restrict__ W,
                                                          const IDX *__restrict__ colp,
                                                          const float2 *__restrict__ F, int ns,
                                                          Part4 *__restrict__ part,
                                                          const long long *__restrict__ srp = nullptr) {
  extern __shared__ float2 Fs[];
  if (SMEMF) {
    const int nsp = DENSE ? (ns + kEntryPad - 1) / kEntryPad * kEntryPad : ns;
    for (int i = threadIdx.x; i < 3 * nsp; i += blockDim.x) Fs[i] = i < 3 * ns ? F[i] : make_float2(0.f, 0.f);
    __syncthreads();
  }
  const float2 *__restrict__ Fg = SMEMF ? Fs : F;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long c0 = I.start;
    const int pb0 = DENSE ? (int)(c0 - srp[I.row]) : 0;  // partner of the item's first entry
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int j = lane;
    bool full = j + 96 < I.len;
    float2 w[4];
    unsigned p[4];
    auto load = [&](int at, float2 (&wv)[4], unsigned (&pv)[4]) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        wv[k] = __ldcs(W + c0 + at + 32 * k);
        pv[k] = DENSE ? (unsigned)(pb0 + at + 32 * k) : (unsigned)__ldcs(colp + c0 + at + 32 * k) & 0xFFFFFFu;
      }
    };
    if (RP && full) load(j, w, p);
    while (full) {
      const bool nfull = j + 128 + 96 < I.len;
      float2 wn[4];
      unsigned pn[4];
      if (RP) {
        if (nfull) load(j + 128, wn, pn);
      } else {
        load(j, w, p);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) tr_mac3<LAZY, !SMEMF>(acc, Fg + 3 * p[k], w[k]);
      if (RP && nfull) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          w[k] = wn[k];
          p[k] = pn[k];
        }
      }
      j += 128;
      full = nfull;
    }
    for (; j < I.len; j += 32) {
      const float2 wk = __ldcs(W + c0 + j);
      const unsigned pk = DENSE ? (unsigned)(pb0 + j) : (unsigned)__ldcs(colp + c0 + j) & 0xFFFFFFu;
      tr_mac3<LAZY, !SMEMF>(acc, Fg + 3 * pk, wk);
    }
    const double X = warp_sum_ff(make_float2(acc[0], acc[1]));
    const double Y = warp_sum_ff(make_float2(acc[2], acc[3]));
    const double Z = warp_sum_ff(make_float2(acc[4], acc[5]));
    if (lane == 0) part[it] = make_part4(X, Y, Z, 0.0);
  }
}

// Transport sweep over complete rows in row blocks.  A warp takes RB consecutive rows and one
// segment of their partner states, consecutive lanes on consecutive partners: each partner's F
// (three float-float values, read from shared memory) serves the RB rows, and each weight row is
// read once, 256 contiguous bytes per warp and trip.  The weights reach shared memory through a
// per-warp ring of D trips filled by asynchronous copies (cp.async, 8 bytes per lane and row, each
// lane reading back only what it copied itself), so D - 1 trips of loads stay in flight without
// holding registers.  Work items are numbered segment-major (item = seg * nblk + block): in a
// launch of one wave a CTA's warps need F only over one or two segments, and only that range is
// staged.  Each lane adds at most seglen / 32 <= 64 terms per sum with lazy renormalisation; the
// warp's RB x 3 sums are reduce-scattered over its lanes (full float-float additions), and the
// (row, segment) totals go to part[row * nseg + seg] in FP64, which the transport finaliser adds
// over a row's nseg segments.  W + srp[r] is row r's first weight, its partners in state order
// (complete rows).  Shared memory: F of up to ns states (24 bytes each), then the rings.
constexpr int kTrRows = 4;          // rows per warp item
constexpr int kTrSegMax = 2048;     // longest segment (64 terms per lane)
constexpr int kTrThreads = 768;     // one CTA per SM, 24 warps, up to 85 registers a thread
constexpr int kTrRing = 4;          // trips per warp ring (three in flight)
__host__ __device__ constexpr size_t tr_rows_ring_offset(int ns) {
  return ((size_t)ns * 3 * sizeof(float2) + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t tr_rows_smem(int ns) {
  return tr_rows_ring_offset(ns) + (size_t)(kTrThreads / 32) * kTrRing * kTrRows * 32 * sizeof(float2);
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int RB>
__global__ void __launch_bounds__(kTrThreads, 1) k_stream_tr_rows(const float2 *__restrict__ W,
                                                                  const long long *__restrict__ srp,
                                                                  const float2 *__restrict__ F, int ns, int nseg,
                                                                  int seglen, Part4 *__restrict__ part) {
  static_assert(RB % 2 == 0, "rows are reduced in pairs");
  constexpr int D = kTrRing;
  extern __shared__ __align__(128) unsigned char trsm[];
  float2 *Fs = (float2 *)trsm;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float2 *ring = (float2 *)(trsm + tr_rows_ring_offset(ns)) + (size_t)wib * D * RB * 32 + lane;  // [D][RB][32]
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int nblk = (ns + RB - 1) / RB, nit = nblk * nseg;
  const int wpb = (int)(blockDim.x >> 5), i0 = (int)blockIdx.x * wpb;
  // the partner range this CTA reads: its items' segments when the launch is one wave
  int cbeg = 0, cend = ns;
  if (nit <= nwarps) {
    if (i0 >= nit) return;
    const int i1 = min(nit, i0 + wpb) - 1;
    cbeg = (i0 / nblk) * seglen;
    cend = min(ns, (i1 / nblk + 1) * seglen);
  }
  for (int i = threadIdx.x; i < 3 * (cend - cbeg); i += blockDim.x) Fs[i] = F[3 * cbeg + i];
  __syncthreads();
  for (int it = i0 + wib; it < nit; it += nwarps) {
    const int seg = it / nblk, r0 = (it - seg * nblk) * RB;
    const int cs = seg * seglen + lane, c1 = min(ns, (seg + 1) * seglen);
    const int ntrip = (c1 - seg * seglen + 31) / 32;
    // rows past the end read the last row again (their sums are not written)
    const long long b0 = srp[r0];
    const float2 *__restrict__ W0 = W + b0;
    int ro[RB];  // row offsets from the first row, in entries
#pragma unroll
    for (int i = 0; i < RB; ++i) ro[i] = (int)(srp[min(r0 + i, ns - 1)] - b0);
    auto fill = [&](int t) {  // this lane's weights of trip t into ring slot t % D (one group per call)
      const int c = cs + 32 * t;
      if (t < ntrip && c < c1) {
#pragma unroll
        for (int i = 0; i < RB; ++i) cp_async8(ring + ((t % D) * RB + i) * 32, W0 + ro[i] + c);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int t = 0; t < D - 1; ++t) fill(t);
    float acc[RB][6];
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[i][k] = 0.f;
    for (int t = 0; t < ntrip; ++t) {
      fill(t + D - 1);
      cp_async_wait<D - 1>();  // trip t's group is complete
      const int c = cs + 32 * t;
      if (c < c1) {
        const float2 *Fp = Fs + 3 * (c - cbeg);
        const float2 fx = Fp[0], fy = Fp[1], fz = Fp[2];
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const float2 w = ring[((t % D) * RB + i) * 32];
          ff_mac_lazy(acc[i][0], acc[i][1], fx, w.x, w.y);
          ff_mac_lazy(acc[i][2], acc[i][3], fy, w.x, w.y);
          ff_mac_lazy(acc[i][4], acc[i][5], fz, w.x, w.y);
        }
      }
    }
    cp_async_wait<0>();  // nothing of this item left in flight before the ring is reused
    // two rows (six sums, two zeros) at a time: lanes 4k .. 4k + 3 end with sum k of the pair
#pragma unroll
    for (int q = 0; q < RB / 2; ++q) {
      float2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int i = 2 * q + m / 3, k = m % 3;
        v[m] = m < 6 ? make_float2(acc[i][2 * k], acc[i][2 * k + 1]) : make_float2(0.f, 0.f);
      }
      ff_reduce_scatter<8, 16>(v, lane);
      const int m = lane >> 2, row = r0 + 2 * q + m / 3;
      if ((lane & 3) == 0 && m < 6 && row < ns)
        (&part[(long long)row * nseg + seg].x)[m % 3] = ff_to_double(v[0].x, v[0].y);
    }
  }
}

// ------------------------------------------------------------ mixed precision (FP32 / BF16 / FP16 |g|^2)
//
// The literal per-channel form of Eq. 2 in FP32: stream |g|^2 (FP32, BF16 or scaled FP16) and the packed
// (partner, branch) word; gather the partner's 16-byte record (energy and occupation, each as
// a hi + lo pair, and its padded grid index) from shared memory and (hbar w, N) from an FP32
// table in L2; evaluate the two Gaussians with ex2 and F_abs / F_em in
// registers; accumulate each lane with Kahan compensation.  Partials, finalisers, RK4 and
// transport stay FP64.
//
// The occupations enter at FP32 precision plus a first-order correction from their low
// parts.  Rounding f to FP32 alone would perturb every term of a row by the same relative
// amount (and every term with partner p likewise), an error that does not average out over
// the row: d I_s / d f_s = -1/tau_s is large while I_s itself shrinks as f relaxes.  The
// correction removes it at the cost of a few FMAs per channel.
//
// Phonon table index without a modulo: the table is laid out on a padded grid of radix
// R_i = 2 N_i (R_i = 1 when N_i = 1), indexed by D_i = j_p,i - j_s,i + N_i in [1, 2 N_i).
// With L(k) = (j1 R2 + j2) R3 + j3 the index is L(k_p) - L(k_s) + L(N1, N2, N3), so each
// state carries L(k) * nmodes and a channel needs two integer adds.  The Gaussian
// normalisation 1/(sqrt(2 pi) sigma) is applied once by the finaliser.

struct GGeom {
  const uint32_t *col;
  const float2 *tabp;  // padded [R1 R2 R3][nmodes] (hbar w, N)
  int cpad;            // L(N1, N2, N3) * nmodes
  float k2;            // -log2(e) / (2 sigma^2)
};

// Per-state record of the mixed-precision sweeps (16 bytes, one shared-memory load):
//   .x  eps hi (FP32)
//   .y  eps lo rounded to 12 significand bits; its low 11 bits hold bits 16..26 of L * nmodes
//   .z  f hi (FP32)
//   .w  high half: f lo as BF16; low half: bits 0..15 of L * nmodes
// eps lo keeps eps to about 2^-36 relative (1e-11 eV at 1 eV, far inside sigma^2 / |x +- w|)
// and f lo keeps f to about 2^-33; L * nmodes must stay below 2^27.
constexpr int kRecLnmBits = 27;
__device__ __forceinline__ int rec_lnm(uint4 r) { return (int)((r.w & 0xFFFFu) | ((r.y & 0x7FFu) << 16)); }
__device__ __forceinline__ float rec_eps_lo(uint4 r) { return __uint_as_float(r.y & 0xFFFFF800u); }
__device__ __forceinline__ float rec_f_lo(uint4 r) { return __uint_as_float(r.w & 0xFFFF0000u); }
// f hi and the BF16 f lo; the grid-index bits in the low half of .w are left in place
__device__ __forceinline__ void rec_set_f(uint4 *rec, double f) {
  const float h = __double2float_rn(f);
  const float l = __double2float_rn(f - (double)h);
  reinterpret_cast<float *>(rec)[2] = h;
  reinterpret_cast<unsigned short *>(rec)[7] = __bfloat16_as_ushort(__float2bfloat16_rn(l));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float t) {
  const float y = __fsub_rn(t, comp);
  const float s2 = __fadd_rn(sum, y);
  comp = __fsub_rn(__fsub_rn(s2, sum), y);
  sum = s2;
}

// One channel: g2 * [G_a F_abs + G_e F_em] (MODE_COLL) or g2 * [G_a (N+f_p) + G_e (N+1-f_p)]
// without the Gaussian normalisation.  ss/sp: row and partner records; base = cpad - L_s nmodes.
template <int MODE>
__device__ __forceinline__ float g_term(const GGeom &g, uint4 ss, uint4 sp, uint32_t cw, int base, float g2) {
  const float2 t = __ldg(g.tabp + (base + rec_lnm(sp) + (int)(cw >> 24)));
  const float dh = __fsub_rn(__uint_as_float(ss.x), __uint_as_float(sp.x));
  const float dl = __fsub_rn(rec_eps_lo(ss), rec_eps_lo(sp));
  const float a = (dh + t.x) + dl;  // x + w
  const float e = (dh - t.x) + dl;  // x - w
  const float Ga = ex2_approx(a * a * g.k2);
  const float Ge = ex2_approx(e * e * g.k2);
  const float fs = __uint_as_float(ss.z), fp = __uint_as_float(sp.z), N = t.y;
  const float fpl = rec_f_lo(sp);
  const float S = Ga + Ge, Dg = Ga - Ge, GN = S * N;
  if (MODE == MODE_COLL) {
    // u = f_s [GN + G_e] - f_p [GN + G_a] + f_s f_p (G_a - G_e), evaluated as
    // F_abs = (f_s - f_p) N - B,  F_em = (f_s - f_p) N + A,  A = f_s (1-f_p), B = (1-f_s) f_p
    const float P = fs * fp;
    const float A = fs - P, B = fp - P;
    const float DN = (fs - fp) * N;
    float u = S * DN;
    u = fmaf(Ge, A, u);
    u = fmaf(-Ga, B, u);
    // low parts of f: du/df_s = GN + G_e + f_p (G_a - G_e), du/df_p = -(GN + G_a) + f_s (G_a - G_e)
    const float Xc = fmaf(fp, Dg, GN + Ge);
    const float Yc = fmaf(-fs, Dg, GN + Ga);
    u = fmaf(rec_f_lo(ss), Xc, u);
    u = fmaf(-fpl, Yc, u);
    return g2 * u;
  }
  return g2 * fmaf(Dg, fpl, fmaf(Dg, fp, GN + Ge));
}

// 16-bit |g|^2 storage: BF16, or FP16 holding |g|^2 times a power of two (the H16 variant;
// the factor is taken out with the collision prefactor).  Two packed values (the lower
// address in the low half) as FP32:
template <typename G2T>
__device__ __forceinline__ float2 g2_pair16(unsigned w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}
template <>
__device__ __forceinline__ float2 g2_pair16<__half>(unsigned w) {
  return make_float2(__half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu))),
                     __half2float(__ushort_as_half((unsigned short)(w >> 16))));
}
// |g|^2 (times the storage factor) in the storage type, rounded to nearest
template <typename G2T>
__device__ __forceinline__ void g2_store(G2T *__restrict__ out, size_t i, double v);
template <>
__device__ __forceinline__ void g2_store<float>(float *__restrict__ out, size_t i, double v) { out[i] = __double2float_rn(v); }
template <>
__device__ __forceinline__ void g2_store<__nv_bfloat16>(__nv_bfloat16 *__restrict__ out, size_t i, double v) {
  out[i] = __double2bfloat16(v);
}
template <>
__device__ __forceinline__ void g2_store<__half>(__half *__restrict__ out, size_t i, double v) { out[i] = __double2half(v); }

// four consecutive |g|^2 values as FP32 (a 16-byte FP32 load or an 8-byte 16-bit load)
template <typename G2T>
__device__ __forceinline__ float4 load_g2x4(const G2T *__restrict__ g2v, long long q) {
  if (sizeof(G2T) == 4) return __ldcs((const float4 *)g2v + q);
  const uint2 v = __ldcs((const uint2 *)g2v + q);
  const float2 a = g2_pair16<G2T>(v.x), b = g2_pair16<G2T>(v.y);
  return make_float4(a.x, a.y, b.x, b.y);
}

// part[item].x = sum over the item of the channel terms above.
template <int MODE, typename G2T>
__global__ void __launch_bounds__(512) k_stream_g(const Item *__restrict__ items, int nitems, GGeom g,
                                                  const G2T *__restrict__ g2v, const uint4 *__restrict__ gstate,
                                                  int ns, Part4 *__restrict__ part) {
  extern __shared__ uint4 gs[];
  for (int i = threadIdx.x; i < ns; i += blockDim.x) gs[i] = gstate[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint4 *__restrict__ col4 = (const uint4 *)g.col;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const uint4 ss = gs[I.row];
    const int base = g.cpad - rec_lnm(ss);
    const long long g0 = I.start >> 2;
    const int ng = I.len >> 2;
    float sum = 0.f, comp = 0.f;
    // software pipeline: the next group's stream words are in flight while this group's
    // partner records and phonon-table entries are gathered and evaluated
    uint4 c = make_uint4(0u, 0u, 0u, 0u);
    float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < ng) {
      c = __ldcs(col4 + g0 + lane);
      gv = load_g2x4(g2v, g0 + lane);
    }
    for (int q = lane; q < ng; q += 32) {
      uint4 cn = make_uint4(0u, 0u, 0u, 0u);
      float4 gn = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q + 32 < ng) {
        cn = __ldcs(col4 + g0 + q + 32);
        gn = load_g2x4(g2v, g0 + q + 32);
      }
      const float t0 = g_term<MODE>(g, ss, gs[c.x & 0xFFFFFFu], c.x, base, gv.x);
      const float t1 = g_term<MODE>(g, ss, gs[c.y & 0xFFFFFFu], c.y, base, gv.y);
      const float t2 = g_term<MODE>(g, ss, gs[c.z & 0xFFFFFFu], c.z, base, gv.z);
      const float t3 = g_term<MODE>(g, ss, gs[c.w & 0xFFFFFFu], c.w, base, gv.w);
      kahan_add(sum, comp, t0);
      kahan_add(sum, comp, t1);
      kahan_add(sum, comp, t2);
      kahan_add(sum, comp, t3);
      c = cn;
      gv = gn;
    }
    const double v = warp_sum((double)sum - (double)comp);
    if (lane == 0) part[it] = make_part4(v, 0.0, 0.0, 0.0);
  }
}

// The same sweep with consecutive lanes on consecutive channels: a warp's 32 channels share
// about 32/nmodes partners, so the partner-record and phonon-table gathers touch few banks and
// sectors; |g|^2 and the index words stay coalesced.  Four channels per lane per trip.
template <typename G2T>
__device__ __forceinline__ float g2_at(const G2T *__restrict__ g2v, long long i);
template <>
__device__ __forceinline__ float g2_at<float>(const float *__restrict__ g2v, long long i) { return __ldcs(g2v + i); }
template <>
__device__ __forceinline__ float g2_at<__nv_bfloat16>(const __nv_bfloat16 *__restrict__ g2v, long long i) {
  return __uint_as_float((unsigned)__ldcs((const unsigned short *)g2v + i) << 16);
}
template <>
__device__ __forceinline__ float g2_at<__half>(const __half *__restrict__ g2v, long long i) {
  return __half2float(__ushort_as_half(__ldcs((const unsigned short *)g2v + i)));
}

// L2 prefetch of the 128-channel trip that starts at channel c (inside the item): lanes 0-3
// take the four 128-byte lines of the index words, the next lanes those of |g|^2.
template <typename G2T>
__device__ __forceinline__ void prefetch_trip(const uint32_t *__restrict__ col, const G2T *__restrict__ g2v,
                                              long long c, int avail, int lane) {
  constexpr int kG2Lines = (int)(128 * sizeof(G2T) / 128);
  const void *a = nullptr;
  if (lane < 4) {
    if (32 * lane < avail) a = col + c + 32 * lane;
  } else if (lane < 4 + kG2Lines) {
    const int k = lane - 4, per = 128 / (int)sizeof(G2T);
    if (per * k < avail) a = g2v + c + per * k;
  }
  if (a) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// Stream words and |g|^2 of one 128-channel trip (lane takes channels j, j+32, j+64, j+96).
template <typename G2T>
__device__ __forceinline__ void load_trip(const uint32_t *__restrict__ col, const G2T *__restrict__ g2v, long long c,
                                          unsigned (&cw)[4], float (&gv)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    cw[k] = __ldcs(col + c + 32 * k);
    gv[k] = g2_at(g2v, c + 32 * k);
  }
}

// PF > 0: each trip first prefetches, into L2, the trip PF ahead in the same item.
// RP: the next trip's stream words are loaded into registers before this trip's gathers and
// arithmetic, so that their HBM latency overlaps this trip (used with NT = 1024: one CTA per
// SM, which leaves most of L1 to the phonon-table gathers and 64 registers per thread).
template <int MODE, typename G2T, int PF, int NT, bool RP>
__global__ void __launch_bounds__(NT, NT == 512 ? 3 : 1) k_stream_g_lane(const Item *__restrict__ items, int nitems, GGeom g,
                                                         const G2T *__restrict__ g2v,
                                                         const uint4 *__restrict__ gstate, int ns,
                                                         Part4 *__restrict__ part) {
  extern __shared__ uint4 gsl[];
  for (int i = threadIdx.x; i < ns; i += blockDim.x) gsl[i] = gstate[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const uint4 ss = gsl[I.row];
    const int base = g.cpad - rec_lnm(ss);
    const long long c0 = I.start;
    float sum = 0.f, comp = 0.f;
    if (PF > 0)
      for (int k = 1; k < PF; ++k)
        if (128 * k < I.len) prefetch_trip(g.col, g2v, c0 + 128 * k, I.len - 128 * k, lane);
    int j = lane;
    bool full = j + 96 < I.len;
    unsigned cw[4] = {0u, 0u, 0u, 0u};
    float gv[4] = {0.f, 0.f, 0.f, 0.f};
    if (RP && full) load_trip(g.col, g2v, c0 + j, cw, gv);
    while (full) {
      if (PF > 0) {
        const int nx = j - lane + 128 * PF;
        if (nx < I.len) prefetch_trip(g.col, g2v, c0 + nx, I.len - nx, lane);
      }
      const bool nfull = j + 128 + 96 < I.len;
      unsigned cn[4];
      float gn[4];
      if (RP) {
        if (nfull) load_trip(g.col, g2v, c0 + j + 128, cn, gn);
      } else {
        load_trip(g.col, g2v, c0 + j, cw, gv);
      }
      float t[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) t[k] = g_term<MODE>(g, ss, gsl[cw[k] & 0xFFFFFFu], cw[k], base, gv[k]);
      // one compensated add per trip; the four-term partial sum rounds like any term
      kahan_add(sum, comp, (t[0] + t[1]) + (t[2] + t[3]));
      if (RP && nfull) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          cw[k] = cn[k];
          gv[k] = gn[k];
        }
      }
      j += 128;
      full = nfull;
    }
    for (; j < I.len; j += 32) {
      const unsigned c = __ldcs(g.col + c0 + j);
      kahan_add(sum, comp, g_term<MODE>(g, ss, gsl[c & 0xFFFFFFu], c, base, g2_at(g2v, c0 + j)));
    }
    const double v = warp_sum((double)sum - (double)comp);
    if (lane == 0) part[it] = make_part4(v, 0.0, 0.0, 0.0);
  }
}

// Dense pair-major form of the mixed-precision sweep.  |g|^2 is stored in one slot per
// (row s, partner p, branch nu): g2d[(s * npp + p) * nm + nu], zero where the channel does not
// exist, so no index is streamed; a pair's branches are contiguous (a few vector loads at fixed
// offsets) and a warp's 32 partners one contiguous run.  A lane takes one partner at a time:
// the partner record, the energy difference and the occupation products once per pair, then
// the nm branches with their (hbar w, N) from the table row of q = k_p - k_s.  g_term's bracket
// with its first-order low-part corrections is bilinear in (G_a, G_e); collected per pair it is
//   u = G_a (N alpha - gamma') + G_e (N alpha + beta'),   alpha = (f_s - f_p) + (f_s,lo - f_p,lo),
//   delta = f_s,lo f_p + f_p,lo f_s,  beta' = A + f_s,lo - delta,  gamma' = B + f_p,lo - delta
// (A = f_s (1 - f_p), B = (1 - f_s) f_p as g_term forms them), and the rate summand is
// G_a (N + f_p) + G_e (N + 1 - f_p) with f_p = hi + lo: a few operations per branch besides the
// Gaussians.  A lane's nm terms are summed and added to its compensated sum once per pair.  An
// item is a run of partners of one row (I.start = s * npp + first partner); its partial goes to
// part[item].x.  MODE_VJP: the FP32 adjoint's sum, the rate summands of each pair weighted by
// lam_s - lam_p (lam in FP32 after the records in shared memory; see k_stream_g_vjp).
constexpr int kDenseBranches = 6;  // branches whose loads a lane issues together (more: one at a time)
constexpr int kDenseThreads = 1024;  // one CTA per SM (768 threads without spills measured slower)
template <int MODE, typename G2T>
__global__ void __launch_bounds__(kDenseThreads, 1) k_stream_g_dense(const Item *__restrict__ items, int nitems, GGeom g,
                                                            const G2T *__restrict__ g2d, int npp, int nm,
                                                            const uint4 *__restrict__ gstate, int ns,
                                                            Part4 *__restrict__ part,
                                                            const float *__restrict__ lam32 = nullptr) {
  extern __shared__ uint4 gsd[];
  float *lsm = reinterpret_cast<float *>(gsd + ns);  // MODE_VJP
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    gsd[i] = gstate[i];
    if (MODE == MODE_VJP) lsm[i] = lam32[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const int s = I.row;
    const uint4 ss = gsd[s];
    const int base = g.cpad - rec_lnm(ss);
    const int p0 = (int)(I.start - (long long)s * npp);
    const G2T *__restrict__ gr = g2d + (size_t)s * npp * nm;
    const float fs = __uint_as_float(ss.z), fsl = rec_f_lo(ss), es = __uint_as_float(ss.x), esl = rec_eps_lo(ss);
    const float ls = MODE == MODE_VJP ? lsm[s] : 0.f;
    float sum = 0.f, comp = 0.f;
    for (int j = lane; j < I.len; j += 32) {
      const int p = p0 + j;
      if (p >= ns) break;  // the row's padding slots (zero |g|^2, no record)
      const uint4 sp = gsd[p];
      const float dh = __fsub_rn(es, __uint_as_float(sp.x));
      const float dl = __fsub_rn(esl, rec_eps_lo(sp));
      const float fp = __uint_as_float(sp.z), fpl = rec_f_lo(sp);
      float alpha, betap, gammap;  // pair constants of the collision bracket (or of the rate summand)
      if (MODE == MODE_COLL) {
        const float P = fs * fp, A = fs - P, B = fp - P;
        const float delta = fmaf(fsl, fp, fpl * fs);
        alpha = (fs - fp) + (fsl - fpl);
        betap = (A + fsl) - delta;
        gammap = (B + fpl) - delta;
      } else {
        alpha = fp + fpl;  // f_p
        betap = 1.f - alpha;
        gammap = 0.f;
      }
      const float2 *__restrict__ tr = g.tabp + (base + rec_lnm(sp));
      auto term = [&](float gv, float2 t) {
        const float a = (dh + t.x) + dl;  // x + w
        const float e = (dh - t.x) + dl;  // x - w
        const float Ga = ex2_approx(a * a * g.k2);
        const float Ge = ex2_approx(e * e * g.k2);
        float u;
        if (MODE == MODE_COLL) {
          const float na = alpha * t.y;
          u = fmaf(Ge, na + betap, Ga * (na - gammap));
        } else {
          u = fmaf(Ge, t.y + betap, Ga * (t.y + alpha));
        }
        return gv * u;
      };
      float acc = 0.f;
      const G2T *__restrict__ gq = gr + (size_t)p * nm;  // the pair's nm slots
      if (nm <= kDenseBranches) {
        // all of the pair's loads first (|g|^2 from HBM, (hbar w, N) from L1/L2), then the terms
        float gv[kDenseBranches];
        float2 tv[kDenseBranches];
        if ((nm & 1) == 0) {  // even nm: the slots of a pair start 8-byte (FP32) / 4-byte (16-bit) aligned
#pragma unroll
          for (int k = 0; k < kDenseBranches / 2; ++k)
            if (2 * k < nm) {
              if (sizeof(G2T) == 4) {
                const float2 v = __ldcs(reinterpret_cast<const float2 *>(gq) + k);
                gv[2 * k] = v.x;
                gv[2 * k + 1] = v.y;
              } else {
                const float2 v = g2_pair16<G2T>(__ldcs(reinterpret_cast<const unsigned *>(gq) + k));
                gv[2 * k] = v.x;
                gv[2 * k + 1] = v.y;
              }
            }
        } else {
#pragma unroll
          for (int nu = 0; nu < kDenseBranches; ++nu)
            if (nu < nm) gv[nu] = g2_at(gq, nu);
        }
#pragma unroll
        for (int nu = 0; nu < kDenseBranches; ++nu)
          if (nu < nm) tv[nu] = __ldg(tr + nu);
#pragma unroll
        for (int nu = 0; nu < kDenseBranches; ++nu)
          if (nu < nm) acc += term(gv[nu], tv[nu]);
      } else {
        for (int nu = 0; nu < nm; ++nu) acc += term(g2_at(gq, nu), __ldg(tr + nu));
      }
      kahan_add(sum, comp, MODE == MODE_VJP ? (ls - lsm[p]) * acc : acc);
    }
    // float-float tree of (sum, -comp), then one conversion
    const double v = warp_sum_ff(make_float2(sum, -comp));
    if (lane == 0) part[it] = make_part4(v, 0.0, 0.0, 0.0);
  }
}

// g2d[(r * npp + p) * nm + nu] = s2 |g|^2 of the stored channel (r, p, nu) in the storage type
// (round to nearest; s2 a power of two); the array is cleared before, so missing channels keep
// zero slots
template <typename G2T>
__global__ void __launch_bounds__(kBlock) k_dense_g2(const Item *__restrict__ items, int nitems,
                                                     const long long *__restrict__ rp_pad,
                                                     const long long *__restrict__ rp_real,
                                                     const uint32_t *__restrict__ col, const double *__restrict__ g2,
                                                     int nm, int npp, G2T *__restrict__ g2d, double s2) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const int r = I.row;
    const long long off = I.start - rp_pad[r];
    const long long real_len = rp_real[r + 1] - rp_real[r];
    for (int j = lane; j < I.len; j += 32) {
      if (off + j >= real_len) break;
      const long long c = I.start + j;
      const unsigned cw = col[c];
      const size_t slot = ((size_t)r * npp + (cw & 0xFFFFFFu)) * (size_t)nm + (cw >> 24);
      g2_store(g2d, slot, s2 * g2[c]);
    }
  }
}

// FP32 adjoint of the mixed-precision sweep.  With w_c(f_p) = g2 [G_a (N+f_p) + G_e (N+1-f_p)]
// (the rate summand) the VJP of Eq. 2 is  (J^T lam)_x = -c sum_{row x} (lam_x - lam_p) w_c(f_p):
// the coefficient form's c [sum lam_p (P_in + (1-f_p) D) - lam_x sum W] written per channel.
// lam32 holds lam in FP32 (staged in shared memory after the state records).
template <typename G2T>
__global__ void __launch_bounds__(512) k_stream_g_vjp(const Item *__restrict__ items, int nitems, GGeom g,
                                                      const G2T *__restrict__ g2v, const uint4 *__restrict__ gstate,
                                                      const float *__restrict__ lam32, int ns,
                                                      Part4 *__restrict__ part) {
  extern __shared__ uint4 gsv[];
  float *lsm = (float *)(gsv + ns);
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    gsv[i] = gstate[i];
    lsm[i] = lam32[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const uint4 ss = gsv[I.row];
    const float ls = lsm[I.row];
    const int base = g.cpad - rec_lnm(ss);
    float sum = 0.f, comp = 0.f;
    for (int j = lane; j < I.len; j += 32) {
      const unsigned cw = __ldcs(g.col + I.start + j);
      const unsigned p = cw & 0xFFFFFFu;
      const float w = g_term<MODE_RATE>(g, ss, gsv[p], cw, base, g2_at(g2v, I.start + j));
      kahan_add(sum, comp, (ls - lsm[p]) * w);
    }
    const double v = warp_sum((double)sum - (double)comp);
    if (lane == 0) part[it] = make_part4(v, 0.0, 0.0, 0.0);
  }
}

// The cotangent g = wl lam + wm mprev (mprev may be null) in FP32 for k_stream_g_vjp.  With
// tab (one stage of the mixed |g|^2-gradient table, see k_g2grad_g): tab[i] =
// (scale g_i, f_i hi, f_i lo, 1 - f_i) in FP32.
__global__ void k_vjp_prep32(const double *__restrict__ f, const double *__restrict__ lam, double wl,
                             const double *__restrict__ mprev, double wm, int n, float *__restrict__ lam32,
                             double scale, float4 *__restrict__ tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double li = wl * lam[i] + (mprev ? wm * mprev[i] : 0.0);
  lam32[i] = __double2float_rn(li);
  if (tab) {
    const double fi = f[i];
    const float2 fs = ff_split(fi);
    tab[i] = make_float4(__double2float_rn(scale * li), fs.x, fs.y, __double2float_rn(1.0 - fi));
  }
}

// Mixed-precision |g|^2 gradient of NST collision calls at once (one call, or the four stages
// of an RK4 step): grad_g2[c] += sum_j scale lam_s^j [G_a F_abs + G_e F_em](f^j), stored
// channels in CSR order without padding, scale = -(2 pi / hbar N_q) / (sqrt(2 pi) sigma) (the
// Gaussians below are not normalised).  The bracket is
// (G_a + G_e) N (f_s - f_p) + G_e f_s (1-f_p) - G_a (1-f_s) f_p, so with the stage table of
// k_vjp_prep32 (c_j = scale lam^j and f^j per state) and c_j(s) summed over the stages,
//   sum_j c_j [...] = GN W + G_e U - G_a V,  W = sum_j c_j (f_s^j - f_p^j),
//   U = sum_j c_j f_s^j (1 - f_p^j),  V = sum_j c_j (1 - f_s^j) f_p^j,
// with f_s - f_p from the high and low parts of f (it is small where the terms cancel): the
// Gaussians once per channel, FP32 terms, one FP64 update of grad per channel.  NST = 0: W, U, V
// are the FP64 sums over many calls that k_g2acc_g keeps per (state, partner) pair,
// acc[0..2][s ns + p], and the bracket is formed in FP64.
template <int NST>
__global__ void __launch_bounds__(kBlock) k_g2grad_g(const Item *__restrict__ items, int nitems, GGeom g,
                                                     const uint4 *__restrict__ gstate,
                                                     const long long *__restrict__ rp_pad,
                                                     const long long *__restrict__ rp_real,
                                                     const float4 *__restrict__ tab, int ns,
                                                     double *__restrict__ grad,
                                                     const double *__restrict__ acc = nullptr) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const int r = I.row;
    const uint4 ss = __ldg(gstate + r);
    const int base = g.cpad - rec_lnm(ss);
    const long long off = I.start - rp_pad[r];
    const long long real_len = rp_real[r + 1] - rp_real[r];
    const long long len = real_len - off < I.len ? real_len - off : I.len;  // stored channels of the item
    double *__restrict__ gr = grad + rp_real[r] + off;
    float4 rs[NST > 0 ? NST : 1];  // (c, f hi, f lo, c f)
    float rb[NST > 0 ? NST : 1];   // c (1 - f)
#pragma unroll
    for (int j = 0; j < NST; ++j) {
      const float4 t = tab[(long long)j * ns + r];
      rs[j] = make_float4(t.x, t.y, t.z, t.x * t.y);
      rb[j] = t.x * t.w;
    }
    for (int k = lane; k < len; k += 32) {
      const unsigned cw = g.col[I.start + k];
      const unsigned p = cw & 0xFFFFFFu;
      const uint4 sp = __ldg(gstate + p);
      const float2 t = __ldg(g.tabp + (base + rec_lnm(sp) + (int)(cw >> 24)));
      const float dh = __fsub_rn(__uint_as_float(ss.x), __uint_as_float(sp.x));
      const float dl = __fsub_rn(rec_eps_lo(ss), rec_eps_lo(sp));
      const float xa = (dh + t.x) + dl;  // x + w
      const float xe = (dh - t.x) + dl;  // x - w
      const float Ga = ex2_approx(xa * xa * g.k2);
      const float Ge = ex2_approx(xe * xe * g.k2);
      const float GN = (Ga + Ge) * t.y;
      if (NST == 0) {
        const long long npair = (long long)ns * ns, q = (long long)r * ns + p;
        gr[k] += fma((double)GN, acc[q], fma((double)Ge, acc[npair + q], -(double)Ga * acc[2 * npair + q]));
        continue;
      }
      float W = 0.f, U = 0.f, V = 0.f;
#pragma unroll
      for (int j = 0; j < NST; ++j) {
        const float4 q = __ldg(tab + (long long)j * ns + p);
        W = fmaf(rs[j].x, __fsub_rn(rs[j].y, q.y) + __fsub_rn(rs[j].z, q.z), W);
        U = fmaf(rs[j].w, q.w, U);
        V = fmaf(rb[j], q.y, V);
      }
      gr[k] += (double)fmaf(GN, W, fmaf(Ge, U, -Ga * V));
    }
  }
}

// Deferred mixed-precision |g|^2 gradient: the NST stages' W, U, V of k_g2grad_g (the same FP32
// terms) for every (state s, partner p) pair, added into FP64 accumulators acc[0..2][s ns + p];
// k_g2grad_g<0> applies them to the channels.  Rows over blockIdx.y, partners over x.
template <int NST>
__global__ void __launch_bounds__(kBlock) k_g2acc_g(const float4 *__restrict__ tab, int ns,
                                                    double *__restrict__ acc) {
  const long long npair = (long long)ns * ns;
  for (int s = blockIdx.y; s < ns; s += gridDim.y) {
    float4 rs[NST];
    float rb[NST];
#pragma unroll
    for (int j = 0; j < NST; ++j) {
      const float4 t = tab[(long long)j * ns + s];
      rs[j] = make_float4(t.x, t.y, t.z, t.x * t.y);
      rb[j] = t.x * t.w;
    }
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ns; p += gridDim.x * blockDim.x) {
      float W = 0.f, U = 0.f, V = 0.f;
#pragma unroll
      for (int j = 0; j < NST; ++j) {
        const float4 q = __ldg(tab + (long long)j * ns + p);
        W = fmaf(rs[j].x, __fsub_rn(rs[j].y, q.y) + __fsub_rn(rs[j].z, q.z), W);
        U = fmaf(rs[j].w, q.w, U);
        V = fmaf(rb[j], q.y, V);
      }
      const long long i = (long long)s * ns + p;
      acc[i] += (double)W;
      acc[npair + i] += (double)U;
      acc[2 * npair + i] += (double)V;
    }
  }
}

// s2 |g|^2 in the storage type of the mixed-precision variants (round to nearest; s2 is a
// power of two, 1 but for FP16).  For FP16, a value that overflows sets *err = kErrG2Range and
// a nonzero value below FP16's smallest normal number (2^-14: it would keep fewer than 11
// significand bits, or none) sets *err = kErrG2Small.
constexpr int kErrG2Range = 16;
constexpr int kErrG2Small = 17;
template <typename G2T>
__global__ void k_cvt_g2(const double *__restrict__ g2, long long n, G2T *__restrict__ out, double s2,
                         int *__restrict__ err) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = s2 * g2[i];
    g2_store(out, (size_t)i, v);
    if (std::is_same<G2T, __half>::value) {
      if (fabs(v) >= 65520.0) *err = kErrG2Range;  // rounds to FP16 infinity
      else if (v != 0.0 && fabs(v) < 0x1p-14) *err = kErrG2Small;  // subnormal or zero in FP16
    }
  }
}

// Per-state records of the mixed-precision sweep (layout above rec_lnm); f is written per stage.
__global__ void k_gstate_init(const double *__restrict__ eps, const short4 *__restrict__ kc, int n, int R2, int R3,
                              int nmodes, uint4 *__restrict__ gstate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 e = ff_split(eps[i]);
  const short4 k = kc[i];
  const unsigned L = (unsigned)((((int)k.x * R2 + (int)k.y) * R3 + (int)k.z) * nmodes);
  const unsigned lo = (__float_as_uint(e.y) + 0x400u) & 0xFFFFF800u;  // 12 significand bits, rounded
  gstate[i] = make_uint4(__float_as_uint(e.x), lo | ((L >> 16) & 0x7FFu), 0u, L & 0xFFFFu);
}

// Padded phonon table: entry (D1, D2, D3, nu) holds (hbar w, N) in FP32 for
// q = (D_i - N_i) mod N_i.  The energy needs no low part: its FP32 rounding (below 2e-9 eV
// for hbar w < 0.06 eV) perturbs each Gaussian by under 1e-6 of itself, pseudo-randomly
// across (q, nu), well below the FP32 error of the terms.
__global__ void k_tab_padded(const double2 *__restrict__ tab, int N1, int N2, int N3, int R1, int R2, int R3,
                             int nmodes, float2 *__restrict__ out) {
  const long long n = (long long)R1 * R2 * R3 * nmodes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int nu = (int)(i % nmodes);
    long long r = i / nmodes;
    const int D3 = (int)(r % R3);
    r /= R3;
    const int D2 = (int)(r % R2);
    const int D1 = (int)(r / R2);
    const int q1 = ((D1 - (R1 > 1 ? N1 : 0)) % N1 + N1) % N1;
    const int q2 = ((D2 - (R2 > 1 ? N2 : 0)) % N2 + N2) % N2;
    const int q3 = ((D3 - (R3 > 1 ? N3 : 0)) % N3 + N3) % N3;
    const double2 wN = tab[((long long)(q1 * N2 + q2) * N3 + q3) * nmodes + nu];
    out[i] = make_float2(__double2float_rn(wN.x), __double2float_rn(wN.y));
  }
}

// f into the records (the stage input of the mixed-precision sweep)
__global__ void k_gstate_f(const double *__restrict__ f, int n, uint4 *__restrict__ gstate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rec_set_f(gstate + i, f[i]);
}

// ------------------------------------------------------------ adjoint (reverse mode)
//
// VJP of the collision integral.  With I_s = c sum_{row s} [f_p P_in + f_s f_p D - f_s P_out]
// and the reverse channel of every channel in the list (P_in <-> P_out, D -> -D), the
// transposed sum over the channels whose partner is x becomes a sum over row x itself:
//   (J^T lam)_x = c [ sum_{row x} lam_p (P_in + (1 - f_p) D) + lam_x (B_x - R_x) ],
//   B_x = sum_{row x} f_p D.
// So the adjoint is another segmented gather over the same stream: no scatter, no atomics.

// The cotangent of one call, g = wl lam + wm mprev (mprev may be null; an RK4 stage's), into
// g and G: G[3i] = g_i, G[3i+1] = g_i f_i, G[3i+2] = f_i as float-float pairs.  With tab (one
// stage of the |g|^2 gradient's table, see k_g2grad): tab[2i] = (a, b), tab[2i+1] =
// (f_i, 1 - f_i), a = scale g_i f_i, b = scale g_i (1 - f_i), all float-float.
__device__ __forceinline__ void vjp_prep_at(int i, double fi, double li, double *__restrict__ g,
                                            float2 *__restrict__ G, double scale, float4 *__restrict__ tab) {
  g[i] = li;
  G[3 * i] = ff_split(li);
  G[3 * i + 1] = ff_split(li * fi);
  G[3 * i + 2] = ff_split(fi);
  if (tab) {
    const double gi = 1.0 - fi, sl = scale * li;
    const float2 a = ff_split(sl * fi), b = ff_split(sl * gi), fs = ff_split(fi), gs = ff_split(gi);
    tab[2 * i] = make_float4(a.x, a.y, b.x, b.y);
    tab[2 * i + 1] = make_float4(fs.x, fs.y, gs.x, gs.y);
  }
}

__global__ void k_vjp_prep(const double *__restrict__ f, const double *__restrict__ lam, double wl,
                           const double *__restrict__ mprev, double wm, int n, double *__restrict__ g,
                           float2 *__restrict__ G, double scale, float4 *__restrict__ tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  vjp_prep_at(i, f[i], wl * lam[i] + (mprev ? wm * mprev[i] : 0.0), g, G, scale, tab);
}

// part[item] = (sum lam_p P_in, sum lam_p D, sum lam_p f_p D, sum f_p D)
template <bool SMEM, typename IDX>
__global__ void __launch_bounds__(kBlock) k_stream_vjp(const Item *__restrict__ items, int nitems,
                                                       const float4 *__restrict__ A4, const float4 *__restrict__ B4,
                                                       const IDX *__restrict__ colp, const float2 *__restrict__ Gg,
                                                       int ns, Part4 *__restrict__ part) {
  extern __shared__ float2 Gsm[];
  if (SMEM) {
    for (int i = threadIdx.x; i < 3 * ns; i += blockDim.x) Gsm[i] = Gg[i];
    __syncthreads();
  }
  const float2 *__restrict__ Gv = SMEM ? Gsm : Gg;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long g0 = I.start >> 2;
    const int ng = I.len >> 2;
    float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f, h3 = 0.f, l3 = 0.f, h4 = 0.f, l4 = 0.f;
    for (int g = lane; g < ng; g += 32) {
      const long long q = g0 + g;
      const uint4 c = partners4(colp, q);
      const float4 a0 = __ldcs(A4 + 2 * q), a1 = __ldcs(A4 + 2 * q + 1);
      const float4 b0 = __ldcs(B4 + 2 * q), b1 = __ldcs(B4 + 2 * q + 1);
      const unsigned p[4] = {c.x, c.y, c.z, c.w};
      const float ah[4] = {a0.x, a0.z, a1.x, a1.z}, al[4] = {a0.y, a0.w, a1.y, a1.w};
      const float bh[4] = {b0.x, b0.z, b1.x, b1.z}, bl[4] = {b0.y, b0.w, b1.y, b1.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 lp = Gv[3 * p[k]], mp = Gv[3 * p[k] + 1], fp = Gv[3 * p[k] + 2];
        ff_mac_lazy(h1, l1, lp, ah[k], al[k]);
        ff_mac_lazy(h2, l2, lp, bh[k], bl[k]);
        ff_mac_lazy(h3, l3, mp, bh[k], bl[k]);
        ff_mac_lazy(h4, l4, fp, bh[k], bl[k]);
      }
    }
    // float-float partials (no FP64 here; the finaliser converts once per state)
    const float2 S1 = warp_reduce_ff(make_float2(h1, l1)), S2 = warp_reduce_ff(make_float2(h2, l2));
    const float2 S3 = warp_reduce_ff(make_float2(h3, l3)), S4 = warp_reduce_ff(make_float2(h4, l4));
    if (lane == 0) {
      float4 *q = reinterpret_cast<float4 *>(part + it);
      q[0] = make_float4(S1.x, S1.y, S2.x, S2.y);
      q[1] = make_float4(S3.x, S3.y, S4.x, S4.y);
    }
  }
}

// The next RK4 stage's cotangent, prepared by the finaliser of the current stage (f null: none):
// g' = wl lam + wm mu with mu this stage's J^T g, into g, the gather table and tab (if not null).
struct VjpNext {
  const double *f, *lam;
  double wl, wm;
  double *g;
  float4 *tab;
};

// mu = J^T g from the float-float partials of k_stream_vjp; out = mu if not null; with acc_out
// also acc_out = acc_in + mu (the running sum of an RK4 step's stage cotangents); nx: see
// VjpNext.  A 256-thread CTA takes SPC states (8 or 32): each warp adds the item partials of
// SPC / 8 states (lanes over the items, then one 32-lane float-float reduce-scatter of their
// 4 values each), and warp 0 does the FP64 arithmetic of the SPC states at once, one lane per
// state.  Few states (small problems) take SPC = 8 for more CTAs in flight.
template <int SPC>
__global__ void __launch_bounds__(256) k_fin_vjp(const int *__restrict__ item_ptr, const Part4 *__restrict__ part,
                                                 int ns, double c, const double *__restrict__ R,
                                                 const double *__restrict__ g, double *__restrict__ out,
                                                 const double *acc_in, double *acc_out,  // acc_in may be acc_out
                                                 VjpNext nx, float2 *__restrict__ G, double scale) {
  constexpr int SPW = SPC / 8, NV = 4 * SPW, LPV = 32 / NV;  // states per warp, values, lanes per value
  __shared__ float2 tot[SPC][4];  // S1..S4 per state
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int base = blockIdx.x * SPC;
  const int r0 = base + lane;
  // warp 0 loads its state's inputs first, so that their latency overlaps the partials'
  double gr = 0.0, Rr = 0.0, ai = 0.0, fn = 0.0, ln = 0.0;
  if (wid == 0 && lane < SPC && r0 < ns) {
    gr = g[r0];
    Rr = R[r0];
    if (acc_out) ai = acc_in[r0];
    if (nx.f) {
      fn = nx.f[r0];
      ln = nx.lam[r0];
    }
  }
  float2 v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < SPW; ++q) {
    const int r = base + SPW * wid + q;
    if (r < ns) {
      for (int i = item_ptr[r] + lane; i < item_ptr[r + 1]; i += 32) {
        const float4 *p = reinterpret_cast<const float4 *>(part + i);
        const float4 a = p[0], b = p[1];
        v[4 * q] = ff_add(v[4 * q], make_float2(a.x, a.y));
        v[4 * q + 1] = ff_add(v[4 * q + 1], make_float2(a.z, a.w));
        v[4 * q + 2] = ff_add(v[4 * q + 2], make_float2(b.x, b.y));
        v[4 * q + 3] = ff_add(v[4 * q + 3], make_float2(b.z, b.w));
      }
    }
  }
  ff_reduce_scatter<NV, 16>(v, lane);
  if ((lane & (LPV - 1)) == 0) {
    const int idx = lane / LPV;  // the top lane bits: (state q, value)
    tot[SPW * wid + (idx >> 2)][idx & 3] = v[0];
  }
  __syncthreads();
  if (wid != 0 || lane >= SPC || r0 >= ns) return;
  const float2 S1 = tot[lane][0], S2 = tot[lane][1], S3 = tot[lane][2], S4 = tot[lane][3];
  const double mu = c * ((ff_to_double(S1.x, S1.y) + ff_to_double(S2.x, S2.y) - ff_to_double(S3.x, S3.y)) +
                         gr * (ff_to_double(S4.x, S4.y) - Rr));
  if (out) out[r0] = mu;
  if (acc_out) acc_out[r0] = ai + mu;
  if (nx.f) vjp_prep_at(r0, fn, nx.wl * ln + nx.wm * mu, nx.g, G, scale, nx.tab);
}

// |g|^2 gradient of NST collision calls at once (one call, or the four stages of an RK4
// step): grad_g2[c] += sum_j -c lam_s^j [G_a F_abs + G_e F_em](f^j) for every stored channel
// c (CSR order without padding).  g2 times the bracket is f_s (1-f_p) P_out - (1-f_s) f_p P_in
// with P_out = P_in + D, so with the stage table of k_vjp_prep (scale -c; per state x and
// stage j: a_j(x), b_j(x), f_x^j and 1 - f_x^j)
//   g2 * sum_j term_j = P_out u - P_in v,   u = sum_j a_j(s) (1 - f_p^j),   v = sum_j b_j(s) f_p^j.
// Here the channel coefficients include g2 (devices without branch merging), so the sum is
// divided by it and channels with g2 = 0 are skipped (k_g2grad_pairs below serves the
// branch-merged devices).  Float-float arithmetic; FP64 for the division and the update.
template <int NST>
__device__ __forceinline__ double g2grad_term(const float4 *__restrict__ rc, const float4 *__restrict__ tab, int ns,
                                              unsigned p, float2 pin, float2 dd) {
  float uh = 0.f, ul = 0.f, vh = 0.f, vl = 0.f;
#pragma unroll
  for (int j = 0; j < NST; ++j) {
    const float4 q = __ldg(tab + 2 * (j * ns + (int)p) + 1);
    ff_mac_lazy(uh, ul, make_float2(rc[j].x, rc[j].y), q.z, q.w);
    ff_mac_lazy(vh, vl, make_float2(rc[j].z, rc[j].w), q.x, q.y);
  }
  const float2 pout = ff_add(pin, dd);
  float th = 0.f, tl = 0.f;
  ff_mac(th, tl, pout, uh, ul);
  ff_mac(th, tl, make_float2(-pin.x, -pin.y), vh, vl);
  return widen_f32(th) + widen_f32(tl);
}

template <int NST, typename IDX>
__global__ void __launch_bounds__(kBlock) k_g2grad(const Item *__restrict__ items, int nitems,
                                                   const long long *__restrict__ rp_pad,
                                                   const long long *__restrict__ rp_real,
                                                   const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                   const IDX *__restrict__ colp, const double *__restrict__ g2,
                                                   const float4 *__restrict__ tab, int ns,
                                                   double *__restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const int r = I.row;
    const long long off = I.start - rp_pad[r];
    const long long real_len = rp_real[r + 1] - rp_real[r];
    const int len = (int)(real_len - off < I.len ? real_len - off : I.len);  // stored channels of the item
    double *__restrict__ gr = grad + rp_real[r] + off;
    const float2 *__restrict__ Ai = A + I.start, *__restrict__ Bi = B + I.start;
    const IDX *__restrict__ ci = colp + I.start;
    float4 rc[NST];
#pragma unroll
    for (int j = 0; j < NST; ++j) rc[j] = tab[2 * (j * ns + r)];
    // two channels per lane per trip: their loads are issued together
    for (int k = lane; k < len; k += 64) {
      const int k1 = k + 32;
      const bool two = k1 < len;
      const unsigned p0 = (unsigned)ci[k] & 0xFFFFFFu, p1 = two ? (unsigned)ci[k1] & 0xFFFFFFu : p0;
      const float2 a0 = Ai[k], b0 = Bi[k];
      const float2 a1 = two ? Ai[k1] : a0, b1 = two ? Bi[k1] : b0;
      const double o0 = gr[k], o1 = two ? gr[k1] : 0.0;
      double t0 = g2grad_term<NST>(rc, tab, ns, p0, a0, b0);
      double t1 = g2grad_term<NST>(rc, tab, ns, p1, a1, b1);
      const double v0 = g2[I.start + k], v1 = two ? g2[I.start + k1] : 1.0;
      t0 = v0 > 0.0 ? t0 / v0 : 0.0;
      t1 = v1 > 0.0 ? t1 / v1 : 0.0;
      gr[k] = o0 + t0;
      if (two) gr[k1] = o1 + t1;
    }
  }
}

// The same gradient on branch-merged devices (coefficients stored without g2), with the
// stage sums u, v computed once per state pair.  A work item is a piece of at most 32
// consecutive sweep entries of a row, one per lane (an entry is the run of pcnt >= 1 channels of
// one partner, from pcstart; padding entries have none), whose channels form one contiguous
// range of the row.  The warp walks that range with coalesced loads, kUnr trips' loads issued
// together; each channel finds the lane of its entry by a binary search over the lanes'
// first-channel offsets and takes u, v from it by shuffles.  NST = 0: u, v come from the pair
// accumulators of the deferred gradient (k_g2acc_pairs), which are cleared once read.
constexpr int kWarpChunk = 32;
constexpr int kGradCtas = 3;  // resident CTAs per SM of k_g2grad_pairs (its persistent grid)
template <int NST, typename IDX>
__global__ void __launch_bounds__(kBlock, kGradCtas) k_g2grad_pairs(const Item *__restrict__ items, int nitems,
                                                                    const IDX *__restrict__ sidx,
                                                                    const long long *__restrict__ pcstart,
                                                                    const uint8_t *__restrict__ pcnt,
                                                                    const long long *__restrict__ rp_pad,
                                                                    const long long *__restrict__ rp_real,
                                                                    const float2 *__restrict__ A,
                                                                    const float2 *__restrict__ B,
                                                                    const float4 *__restrict__ tab, int ns,
                                                                    double *__restrict__ grad,
                                                                    float4 *__restrict__ gacc = nullptr) {
  constexpr int kUnr = 3;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const int r = I.row;
    const long long q = I.start + lane;
    const int m = lane < I.len ? (int)pcnt[q] : 0;
    if (!__any_sync(0xFFFFFFFFu, m > 0)) continue;  // padding only
    double *__restrict__ gr = grad + (rp_real[r] - rp_pad[r]);  // channel position -> unpadded index
    const long long cs = m ? pcstart[q] : 0;
    float uh = 0.f, ul = 0.f, vh = 0.f, vl = 0.f;
    if (m && NST == 0) {
      const float4 a = gacc[q];
      uh = a.x;
      ul = a.y;
      vh = a.z;
      vl = a.w;
      gacc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else if (m) {
      const int p = (int)sidx[q];
#pragma unroll
      for (int j = 0; j < NST; ++j) {
        const float4 rc = tab[2 * (j * ns + r)];
        const float4 t = __ldg(tab + 2 * (j * ns + p) + 1);
        ff_mac_lazy(uh, ul, make_float2(rc.x, rc.y), t.z, t.w);
        ff_mac_lazy(vh, vl, make_float2(rc.z, rc.w), t.x, t.y);
      }
    }
    // real entries precede the padding, so lane 0 holds the first channel of the piece
    const long long cb = __shfl_sync(0xFFFFFFFFu, cs, 0);
    const int rs = m ? (int)(cs - cb) : 0x7FFFFFFF;  // first-channel offset (padding: never owns)
    const int nch = __reduce_max_sync(0xFFFFFFFFu, m ? rs + m : 0);
    const float2 *__restrict__ Ab = A + cb, *__restrict__ Bb = B + cb;
    double *__restrict__ gb = gr + cb;
    for (int o0 = 0; o0 < nch; o0 += 32 * kUnr) {
      float2 pin[kUnr], dd[kUnr];
      double old[kUnr];
#pragma unroll
      for (int k = 0; k < kUnr; ++k) {
        const int o = o0 + 32 * k + lane;
        if (o < nch) {
          pin[k] = Ab[o];
          dd[k] = Bb[o];
          old[k] = gb[o];
        }
      }
#pragma unroll
      for (int k = 0; k < kUnr; ++k) {
        const int o = o0 + 32 * k + lane;
        int own = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int sc = __shfl_sync(0xFFFFFFFFu, rs, own + step);
          if (sc <= o) own += step;
        }
        const float2 u = make_float2(__shfl_sync(0xFFFFFFFFu, uh, own), __shfl_sync(0xFFFFFFFFu, ul, own));
        const float2 v = make_float2(__shfl_sync(0xFFFFFFFFu, vh, own), __shfl_sync(0xFFFFFFFFu, vl, own));
        if (o < nch) {
          const float2 pout = ff_add(pin[k], dd[k]);
          float th = 0.f, tl = 0.f;
          ff_mac(th, tl, pout, u.x, u.y);
          ff_mac(th, tl, make_float2(-pin[k].x, -pin[k].y), v.x, v.y);
          gb[o] = old[k] + (widen_f32(th) + widen_f32(tl));
        }
      }
    }
  }
}

// Deferred |g|^2 gradient of branch-merged devices: the NST stages' sums u, v of every state
// pair (as k_g2grad_pairs forms them) added into the pair's float-float accumulators
// gacc[q] = (u hi, u lo, v hi, v lo); k_g2grad_pairs<0> later applies the accumulated sums to
// the pair's channels once and clears them.  Lane per sweep entry of a piece (padding: none).
template <int NST, typename IDX>
__global__ void __launch_bounds__(kBlock) k_g2acc_pairs(const Item *__restrict__ items, int nitems,
                                                        const IDX *__restrict__ sidx, const uint8_t *__restrict__ pcnt,
                                                        const float4 *__restrict__ tab, int ns,
                                                        float4 *__restrict__ gacc) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long q = I.start + lane;
    if (lane >= I.len || pcnt[q] == 0) continue;
    const int r = I.row, p = (int)sidx[q];
    float uh = 0.f, ul = 0.f, vh = 0.f, vl = 0.f;
#pragma unroll
    for (int j = 0; j < NST; ++j) {
      const float4 rc = tab[2 * (j * ns + r)];
      const float4 t = __ldg(tab + 2 * (j * ns + p) + 1);
      ff_mac_lazy(uh, ul, make_float2(rc.x, rc.y), t.z, t.w);
      ff_mac_lazy(vh, vl, make_float2(rc.z, rc.w), t.x, t.y);
    }
    float4 a = gacc[q];
    const float2 u = ff_add(make_float2(a.x, a.y), make_float2(uh, ul));
    const float2 v = ff_add(make_float2(a.z, a.w), make_float2(vh, vl));
    gacc[q] = make_float4(u.x, u.y, v.x, v.y);
  }
}

// padded g2 from the unpadded CSR order (padding stays zero)
__global__ void k_set_g2(const Item *__restrict__ items, int nitems, const long long *__restrict__ rp_pad,
                         const long long *__restrict__ rp_real, const double *__restrict__ in,
                         double *__restrict__ g2) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long off = I.start - rp_pad[I.row];
    const long long real_len = rp_real[I.row + 1] - rp_real[I.row];
    for (int j = lane; j < I.len; j += 32) {
      const long long k = off + j;
      g2[I.start + j] = k < real_len ? in[rp_real[I.row] + k] : 0.0;
    }
  }
}

// out = a x + b y (y may be null; out may be x or y)
__global__ void k_lincomb(int n, double a, const double *x, double b, const double *y, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

// ------------------------------------------------------------ paper layout (ablation)
//
// The paper's GPU scheme (Sec. "Optimized GPU algorithm", Fig. 2): every physical channel
// is stored once (here: under the state with the lower index), step 2 writes its
// contribution to a per-channel array sc_col, and step 3 lets every state gather +/- sc_col
// over its target list (the signed stargets_sources), with no atomics.  It trades half the
// coefficient storage for an extra write and read of sc_col and a scattered gather.


// sc_col[c] = f_p (P_in + f_s D) - f_s P_out for each stored channel (orientation s -> p);
// its contribution to I_p is -sc_col[c].
template <bool SMEM>
__global__ void __launch_bounds__(kBlock) k_paper_sc(const Item *__restrict__ items, int nitems,
                                                     const float4 *__restrict__ A4, const float4 *__restrict__ B4,
                                                     const uint32_t *__restrict__ hcol,
                                                     const float2 *__restrict__ fg, int ns, float4 *__restrict__ sc4) {
  extern __shared__ float2 fsp[];
  if (SMEM) {
    for (int i = threadIdx.x; i < ns; i += blockDim.x) fsp[i] = fg[i];
    __syncthreads();
  }
  const float2 *__restrict__ fv = SMEM ? fsp : fg;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const float2 fs = fv[I.row];
    const long long g0 = I.start >> 2;
    const int ng = I.len >> 2;
    for (int g = lane; g < ng; g += 32) {
      const long long q = g0 + g;
      const uint4 c = partners4(hcol, q);
      const float4 a0 = __ldcs(A4 + 2 * q), a1 = __ldcs(A4 + 2 * q + 1);
      const float4 b0 = __ldcs(B4 + 2 * q), b1 = __ldcs(B4 + 2 * q + 1);
      const unsigned p[4] = {c.x, c.y, c.z, c.w};
      const float2 pin[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                             make_float2(a1.z, a1.w)};
      const float2 dd[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                            make_float2(b1.z, b1.w)};
      float2 out[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 fp = fv[p[k]];
        const float2 in = ff_mul(fp, ff_add(pin[k], ff_mul(fs, dd[k])));
        const float2 outs = ff_mul(fs, ff_add(pin[k], dd[k]));
        out[k] = ff_add(in, make_float2(-outs.x, -outs.y));
      }
      __stcs(sc4 + 2 * q, make_float4(out[0].x, out[0].y, out[1].x, out[1].y));
      __stcs(sc4 + 2 * q + 1, make_float4(out[2].x, out[2].y, out[3].x, out[3].y));
    }
  }
}

// part[item].x = -(sum of signed sc_col over the item's target entries); entry bit 31 = minus.
__global__ void __launch_bounds__(kBlock) k_paper_gather(const Item *__restrict__ items, int nitems,
                                                         const int *__restrict__ entries,
                                                         const float2 *__restrict__ sc, Part4 *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int4 *__restrict__ e4 = (const int4 *)entries;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long g0 = I.start >> 2;
    const int ng = I.len >> 2;
    float2 acc = make_float2(0.f, 0.f);
    for (int g = lane; g < ng; g += 32) {
      const int4 e = __ldcs(e4 + g0 + g);
      const int ev[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float2 v = __ldg(sc + (ev[k] & 0x7FFFFFFF));
        if (ev[k] < 0) v = make_float2(-v.x, -v.y);
        acc = ff_add(acc, v);
      }
    }
    const double S = warp_sum(ff_to_double(acc.x, acc.y));
    if (lane == 0) part[it] = make_part4(-S, 0.0, 0.0, 0.0);
  }
}

// ------------------------------------------------------------ symmetric tiles (complete rows)
//
// When every row holds every window state, the branch-merged pair matrix is dense, and the
// reverse channels fix its transpose: P_in(p,s) = P_out(s,p) and P_out(p,s) = P_in(s,p). It is
// stored as 64 x 64 tiles of its upper block triangle, (P_in hi, P_in lo, P_out hi, P_out lo)
// per entry. Each off-diagonal tile adds to its rows (partners = its columns) and to its
// columns (partners = its rows):
//   row s:  A += f_p P_in(s,p),   C += f_p P_out(s,p)
//   col p:  A += f_s P_out(s,p),  C += f_s P_in(s,p)
// so each state gets B = C - A = sum f D, as in the row stream. Diagonal tiles hold all
// 64 x 64 entries and add to their rows only. Every tile writes one (A, B) per row and per
// column into tp[state][partner block], so each state receives exactly one partial per block
// of partner states, stored contiguously; the epilogue adds them in block order (no atomics).

constexpr int kTile = 64;

// tc[t][i][j] from the branch-merged coefficients of complete rows (entry (s, p) of row s is
// at srp[s] + p); zero outside the nstate states.
__global__ void k_tiles_fill(const int2 *__restrict__ tiles, int nt, const float2 *__restrict__ coefA,
                             const float2 *__restrict__ coefB, const long long *__restrict__ srp, int ns,
                             float4 *__restrict__ tc) {
  const long long n = (long long)nt * kTile * kTile;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / (kTile * kTile)), k = (int)(e % (kTile * kTile));
    const int2 IJ = tiles[t];
    const int s = IJ.x * kTile + k / kTile, p = IJ.y * kTile + k % kTile;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < ns && p < ns) {
      const long long c = srp[s] + p;
      const float2 a = coefA[c], b = coefB[c];
      const double pin = ff_to_double(a.x, a.y), pout = pin + ff_to_double(b.x, b.y);
      const float2 x = ff_split(pin), y = ff_split(pout);
      v = make_float4(x.x, x.y, y.x, y.y);
    }
    tc[e] = v;
  }
}

// One tile per CTA trip (grid-stride over tiles); thread (ti, tj) takes rows 4ti..4ti+3 and
// columns 4tj..4tj+3 of the tile, so a warp reads two 1 KB row segments per step.  The four
// terms a thread adds per row (per column) use lazily renormalised float-float sums; the 16
// thread partials of a row (column) are then added with full float-float additions.
__global__ void __launch_bounds__(256, 3) k_stream_sym(const int2 *__restrict__ tiles, int nt,
                                                       const float4 *__restrict__ tc,
                                                       const float2 *__restrict__ fg, int ns, int nb,
                                                       float4 *__restrict__ tp) {
  __shared__ float2 fr[kTile], fc[kTile];
  __shared__ float4 red[2][kTile][17];  // [rows | cols][state][thread] (A hi, A lo, C hi, C lo); 17: no bank clash
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int2 IJ = tiles[t];
    const bool diag = IJ.x == IJ.y;
    const int r0 = IJ.x * kTile, c0 = IJ.y * kTile;
    if (tid < kTile) fr[tid] = r0 + tid < ns ? fg[r0 + tid] : make_float2(0.f, 0.f);
    else if (tid < 2 * kTile) fc[tid - kTile] = c0 + tid - kTile < ns ? fg[c0 + tid - kTile] : make_float2(0.f, 0.f);
    __syncthreads();
    float2 fcol[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) fcol[j] = fc[4 * tj + j];
    float rA[4][2], rC[4][2], cA[4][2], cC[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      rA[k][0] = rA[k][1] = rC[k][0] = rC[k][1] = 0.f;
      cA[k][0] = cA[k][1] = cC[k][0] = cC[k][1] = 0.f;
    }
    const float4 *__restrict__ base = tc + (long long)t * kTile * kTile + 4 * tj;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int s = 4 * ti + i;
      const float2 fs = fr[s];
      float4 e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) e[j] = __ldcs(base + s * kTile + j);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ff_mac_lazy(rA[i][0], rA[i][1], fcol[j], e[j].x, e[j].y);
        ff_mac_lazy(rC[i][0], rC[i][1], fcol[j], e[j].z, e[j].w);
        if (!diag) {
          ff_mac_lazy(cA[j][0], cA[j][1], fs, e[j].z, e[j].w);
          ff_mac_lazy(cC[j][0], cC[j][1], fs, e[j].x, e[j].y);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      red[0][4 * ti + k][tj] = make_float4(rA[k][0], rA[k][1], rC[k][0], rC[k][1]);
      red[1][4 * tj + k][ti] = make_float4(cA[k][0], cA[k][1], cC[k][0], cC[k][1]);
    }
    __syncthreads();
    if (tid < 2 * kTile && (tid < kTile || !diag)) {
      const int side = tid >> 6, x = tid & (kTile - 1);
      float2 A = make_float2(0.f, 0.f), C = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int k = 0; k < 16; ++k) {
        const float4 v = red[side][x][k];
        A = ff_add(A, make_float2(v.x, v.y));
        C = ff_add(C, make_float2(v.z, v.w));
      }
      const int st = (side == 0 ? r0 : c0) + x;
      const int blk = side == 0 ? IJ.y : IJ.x;
      tp[(long long)st * nb + blk] = make_float4(A.x, A.y, C.x, C.y);
    }
    __syncthreads();
  }
}

// The same tile sweep with the tiles staged through shared memory by bulk copies
// (cp.async.bulk, completion counted in bytes on an mbarrier): one persistent 256-thread CTA per
// SM; thread 0 keeps kSymStages tiles in flight (each with the float-float f of its row and
// column blocks) while the CTA adds the staged tile.  Thread (ti, tj) takes rows 4ti .. 4ti+3
// and columns tj, tj+16, tj+32, tj+48, so a quarter-warp reads 128 contiguous bytes of a row
// (no bank conflicts).  Row partials are reduced inside the warp by a float-float reduce-scatter
// over the 16 lanes of a row; column partials by one shuffle level into a per-warp table that
// the next iteration combines (double-buffered), so each tile costs one CTA barrier.  Every
// wait is bounded: on a give-up the kernel records it in *err, waits (bounded) for its own
// copies and returns.
constexpr int kSymStages = 3;
constexpr int kSymThreads = 256;
constexpr unsigned kTileBytes = kTile * kTile * sizeof(float4);
constexpr unsigned kSymStageBytes = kTileBytes + 2 * kTile * sizeof(float2);
constexpr size_t kSymColBytes = (size_t)(kSymThreads / 32) * 2 * kTile * sizeof(float2);  // one column table
constexpr size_t kSymBulkSmem = (size_t)kSymStages * kSymStageBytes + 64 + 2 * kSymColBytes;

// the column partials of a finished off-diagonal tile: one (column, A | C) value per lane pair
// (lanes l and l ^ 16 take warps 0-3 and 4-7), renormalised, into tp (slot: the tile's row block,
// slotI; the batched sweep numbers a state's partner blocks within its instance)
__device__ __forceinline__ void sym_columns_out(const float2 *__restrict__ colred, int2 IJ, int slotI, int nb, int lane,
                                                int wid, float4 *__restrict__ tp) {
  constexpr int NW = kSymThreads / 32, WG = NW / 2;
  const int g = lane >> 4;
  const int q = (lane & 15) + 16 * wid;  // 0 .. 127
  const int col = q & (kTile - 1), comp = q >> 6;
  float2 acc = colred[((g * WG) * 2 + comp) * kTile + col];
#pragma unroll
  for (int w = 1; w < WG; ++w) acc = ff_add(acc, colred[((g * WG + w) * 2 + comp) * kTile + col]);
  acc = ff_add(acc, make_float2(__shfl_xor_sync(0xFFFFFFFFu, acc.x, 16), __shfl_xor_sync(0xFFFFFFFFu, acc.y, 16)));
  if (g == 0) ((float2 *)tp)[2 * ((long long)(IJ.y * kTile + col) * nb + slotI) + comp] = acc;
}

__global__ void __launch_bounds__(kSymThreads, 1) k_stream_sym_bulk(const int2 *__restrict__ tiles, int nt,
                                                                     const float4 *__restrict__ tc,
                                                                     const float2 *__restrict__ fg, int ns, int nb,
                                                                     float4 *__restrict__ tp, int *__restrict__ err) {
  constexpr int R = 4, NV = 2 * R;
  extern __shared__ __align__(128) unsigned char ssm[];
  unsigned long long *bars = (unsigned long long *)(ssm + kSymStages * kSymStageBytes);
  int2 *stile = (int2 *)(bars + kSymStages);  // the tile held by each stage
  float2 *colred0 = (float2 *)(ssm + kSymStages * kSymStageBytes + 64);  // 2 x [8 warps][A | C][64 columns]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, tj = tid & 15, ti = tid >> 4;
  const int G = (int)gridDim.x;
  const int nloc = (int)blockIdx.x < nt ? (nt - 1 - (int)blockIdx.x) / G + 1 : 0;
  // the f slices of every stage start as zeros (a copy of a last, partial block leaves the rest)
  for (int i = tid; i < kSymStages * 2 * kTile; i += kSymThreads) {
    float2 *fz = (float2 *)(ssm + (i / (2 * kTile)) * kSymStageBytes + kTileBytes);
    fz[i % (2 * kTile)] = make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    for (int k = 0; k < kSymStages; ++k) mbar_init(bars + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();  // the zeroed f slices before any bulk write to them
  __syncthreads();
  int issued = 0;
  auto issue = [&](int k, int2 IJ) {
    const int s = k % kSymStages;
    const int t = (int)blockIdx.x + k * G;
    stile[s] = IJ;
    unsigned char *buf = ssm + (size_t)s * kSymStageBytes;
    const int nr = min(kTile, ns - IJ.x * kTile), nc = min(kTile, ns - IJ.y * kTile);
    const unsigned br = (unsigned)(nr * sizeof(float2) + 15) / 16 * 16, bc = (unsigned)(nc * sizeof(float2) + 15) / 16 * 16;
    mbar_expect_tx(bars + s, kTileBytes + br + bc);
    const unsigned char *src = (const unsigned char *)(tc + (size_t)t * kTile * kTile);
#pragma unroll
    for (int q = 0; q < 4; ++q) bulk_g2s(buf + q * (kTileBytes / 4), src + q * (kTileBytes / 4), kTileBytes / 4, bars + s);
    bulk_g2s(buf + kTileBytes, fg + (size_t)IJ.x * kTile, br, bars + s);
    bulk_g2s(buf + kTileBytes + kTile * sizeof(float2), fg + (size_t)IJ.y * kTile, bc, bars + s);
  };
  if (tid == 0)
    for (; issued < kSymStages && issued < nloc; ++issued) issue(issued, tiles[(int)blockIdx.x + issued * G]);
  int2 nextIJ = make_int2(0, 0);  // thread 0: descriptor of the next tile to issue, loaded a tile ahead
  if (tid == 0 && issued < nloc) nextIJ = tiles[(int)blockIdx.x + issued * G];
  int2 prevIJ = make_int2(0, 0);  // the previous tile (its columns are combined in this iteration)
  bool ok = true;
  for (int k = 0; k <= nloc; ++k) {
    // thread 0 waits on the mbarrier of tile k (acquire); the CTA barrier publishes the stage
    // to all, and marks the end of tile k-1 (its stage is free, its column table complete)
    const bool have = k < nloc;
    if (!__syncthreads_and(tid == 0 && have ? mbar_wait(bars + k % kSymStages, (unsigned)((k / kSymStages) & 1)) : true)) {
      ok = false;
      break;
    }
    if (tid == 0 && k >= 1 && issued < nloc) {
      fence_proxy_async();  // order the generic reads of tile k-1's stage before its refill
      issue(issued, nextIJ);
      ++issued;
      if (issued < nloc) nextIJ = tiles[(int)blockIdx.x + issued * G];
    }
    if (k >= 1 && prevIJ.x != prevIJ.y)
      sym_columns_out(colred0 + ((k - 1) & 1) * (kSymColBytes / sizeof(float2)), prevIJ, prevIJ.x, nb, lane, wid, tp);
    if (!have) break;
    const int s = k % kSymStages;
    const int2 IJ = stile[s];
    prevIJ = IJ;
    const bool diag = IJ.x == IJ.y;
    const float4 *__restrict__ T = (const float4 *)(ssm + (size_t)s * kSymStageBytes);
    const float2 *__restrict__ fr = (const float2 *)(ssm + (size_t)s * kSymStageBytes + kTileBytes);
    const float2 *__restrict__ fc = fr + kTile;
    float2 fcol[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) fcol[j] = fc[tj + 16 * j];
    // each accumulator's first term is a plain product (no zeroing, no addition)
    float rA[R][2], rC[R][2], cA[4][2], cC[4][2];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int row = ti * R + i;
      const float2 fs = fr[row];
      float4 e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) e[j] = T[row * kTile + tj + 16 * j];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j == 0) {
          ff_prod(rA[i][0], rA[i][1], fcol[j], e[j].x, e[j].y);
          ff_prod(rC[i][0], rC[i][1], fcol[j], e[j].z, e[j].w);
        } else {
          ff_mac_lazy(rA[i][0], rA[i][1], fcol[j], e[j].x, e[j].y);
          ff_mac_lazy(rC[i][0], rC[i][1], fcol[j], e[j].z, e[j].w);
        }
        if (!diag) {
          if (i == 0) {
            ff_prod(cA[j][0], cA[j][1], fs, e[j].z, e[j].w);
            ff_prod(cC[j][0], cC[j][1], fs, e[j].x, e[j].y);
          } else {
            ff_mac_lazy(cA[j][0], cA[j][1], fs, e[j].z, e[j].w);
            ff_mac_lazy(cC[j][0], cC[j][1], fs, e[j].x, e[j].y);
          }
        }
      }
    }
    // rows: the 16 lanes of a half-warp share them; lane tj ends with value idx (row, A | C)
    {
      float2 v[NV];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        v[2 * i] = make_float2(rA[i][0], rA[i][1]);
        v[2 * i + 1] = make_float2(rC[i][0], rC[i][1]);
      }
      ff_reduce_scatter<NV, 8>(v, lane);
      const int idx = ((tj >> 3) & 1) * 4 + ((tj >> 2) & 1) * 2 + ((tj >> 1) & 1);
      if ((tj & 1) == 0) {  // lanes tj and tj ^ 1 hold the same total
        const int row = IJ.x * kTile + ti * R + (idx >> 1);
        ((float2 *)tp)[2 * ((long long)row * nb + IJ.y) + (idx & 1)] = v[0];
      }
    }
    if (!diag) {
      // columns: lanes tj and tj + 16 share them (one level), then the warps (next iteration)
      float2 *colred = colred0 + (k & 1) * (kSymColBytes / sizeof(float2));
      const bool up = lane & 16;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int jk = m >> 1, jo = jk + 2;  // kept / sent column slot
        const float2 a = (m & 1) ? make_float2(cC[jk][0], cC[jk][1]) : make_float2(cA[jk][0], cA[jk][1]);
        const float2 c = (m & 1) ? make_float2(cC[jo][0], cC[jo][1]) : make_float2(cA[jo][0], cA[jo][1]);
        const float2 send = up ? a : c, keep = up ? c : a;
        const float2 w = ff_add(keep, make_float2(__shfl_xor_sync(0xFFFFFFFFu, send.x, 16),
                                                  __shfl_xor_sync(0xFFFFFFFFu, send.y, 16)));
        const int col = tj + 16 * ((up ? 2 : 0) + jk);
        colred[(wid * 2 + (m & 1)) * kTile + col] = w;
      }
    }
  }
  if (!ok) {
    *err = 2;
    if (tid == 0) {  // drain: wait (bounded) for every copy this CTA issued
      for (int k = 0; k < kSymStages; ++k) {
        const int uses = issued / kSymStages + (k < issued % kSymStages ? 1 : 0);
        if (uses > 0) mbar_wait(bars + k, (unsigned)((uses - 1) & 1));
      }
    }
  }
}

// The same float-float tile sweep in half-tiles: the unit of staging is 32 rows x 64 columns of a
// tile (32 KB, contiguous in the tile's row-major layout), so a CTA of 256 threads holds three
// units in shared memory and two CTAs fit on an SM (16 warps, each CTA with its own barrier).
// A CTA takes both halves of each of its tiles in turn: rows are complete within a half (one
// float-float (A, C) partial per row and partner block, as above); the column sums of a tile
// stay in registers across its two halves and go to the per-warp table after the second, and
// the table is combined after the next unit's barrier.  Columns are written only every other
// unit, so one table suffices.  Thread (ti, tj) takes rows 2 ti, 2 ti + 1 of the half and
// columns tj, tj + 16, tj + 32, tj + 48.
constexpr unsigned kHalfTileBytes = kTileBytes / 2;
constexpr unsigned kHalfStageBytes = kHalfTileBytes + (kTile / 2 + kTile) * sizeof(float2);
template <int NST>
constexpr size_t half_smem() {
  return (size_t)NST * kHalfStageBytes + 64 + kSymColBytes;
}

// NST stages per CTA, CPS resident CTAs per SM (3 x 2 or 2 x 3 fit in the SM's shared memory)
// lblk (batched sweep, else null): the block index of each block within its instance, which
// numbers the partial slots; blocks are global otherwise.  rev: take the tile list from its end
// (tile nt - 1 - t in place of t), so that a sweep following one in list order starts on the
// tiles the L2 still holds; the partials do not depend on the order.
template <int NST, int CPS>
__global__ void __launch_bounds__(kSymThreads, CPS) k_stream_sym_half(const int2 *__restrict__ tiles, int nt,
                                                                       const float4 *__restrict__ tc,
                                                                       const float2 *__restrict__ fg, int ns, int nb,
                                                                       float4 *__restrict__ tp, int *__restrict__ err,
                                                                       const int *__restrict__ lblk = nullptr,
                                                                       int rev = 0) {
  constexpr int kHalfStages = NST;
  static_assert(NST >= 2 && NST <= 4, "the ring needs 2..4 stages");
  constexpr int R = 2, NV = 2 * R, HR = kTile / 2;
  extern __shared__ __align__(128) unsigned char ssm[];
  unsigned long long *bars = (unsigned long long *)(ssm + kHalfStages * kHalfStageBytes);
  int2 *stile = (int2 *)(bars + kHalfStages);  // the tile of each stage's unit
  float2 *colred = (float2 *)(ssm + kHalfStages * kHalfStageBytes + 64);  // [8 warps][A | C][64 columns]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, tj = tid & 15, ti = tid >> 4;
  const int G = (int)gridDim.x;
  const int nloc = (int)blockIdx.x < nt ? (nt - 1 - (int)blockIdx.x) / G + 1 : 0;
  const int nunit = 2 * nloc;
  for (int i = tid; i < kHalfStages * (HR + kTile); i += kSymThreads) {
    float2 *fz = (float2 *)(ssm + (i / (HR + kTile)) * kHalfStageBytes + kHalfTileBytes);
    fz[i % (HR + kTile)] = make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    for (int k = 0; k < kHalfStages; ++k) mbar_init(bars + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  __syncthreads();
  // thread 0: units are issued in order; issIJ is the tile being issued, aheadIJ the next one
  int issued = 0;
  auto tix = [&](int k) {  // the CTA's k-th tile
    const int t = (int)blockIdx.x + k * G;
    return rev ? nt - 1 - t : t;
  };
  int2 issIJ = make_int2(0, 0), aheadIJ = make_int2(0, 0);
  if (tid == 0 && nloc > 0) {
    issIJ = tiles[tix(0)];
    if (nloc > 1) aheadIJ = tiles[tix(1)];
  }
  auto issue = [&](int v) {  // unit v = 2 k + h: half h of the CTA's tile k
    const int k = v >> 1, h = v & 1, s = v % kHalfStages;
    if (h == 0 && k > 0) {
      issIJ = aheadIJ;
      if (k + 1 < nloc) aheadIJ = tiles[tix(k + 1)];
    }
    const int t = tix(k);
    stile[s] = issIJ;
    unsigned char *buf = ssm + (size_t)s * kHalfStageBytes;
    const int nr = min(HR, ns - (issIJ.x * kTile + h * HR)), nc = min(kTile, ns - issIJ.y * kTile);
    const unsigned br = nr > 0 ? (unsigned)(nr * sizeof(float2) + 15) / 16 * 16 : 0u;
    const unsigned bc = (unsigned)(nc * sizeof(float2) + 15) / 16 * 16;
    mbar_expect_tx(bars + s, kHalfTileBytes + br + bc);
    const unsigned char *src = (const unsigned char *)(tc + (size_t)t * kTile * kTile) + (size_t)h * kHalfTileBytes;
#pragma unroll
    for (int q = 0; q < 2; ++q) bulk_g2s(buf + q * (kHalfTileBytes / 2), src + q * (kHalfTileBytes / 2), kHalfTileBytes / 2, bars + s);
    if (br) bulk_g2s(buf + kHalfTileBytes, fg + (size_t)issIJ.x * kTile + h * HR, br, bars + s);
    bulk_g2s(buf + kHalfTileBytes + HR * sizeof(float2), fg + (size_t)issIJ.y * kTile, bc, bars + s);
  };
  if (tid == 0)
    for (; issued < kHalfStages && issued < nunit; ++issued) issue(issued);
  int2 prevIJ = make_int2(0, 0);  // the tile of the previous unit
  int prevI = 0;                  // its row block's slot index
  bool ok = true;
  float cA[4][2], cC[4][2];  // column sums of the current tile, carried across its halves
  for (int u = 0; u <= nunit; ++u) {
    const bool have = u < nunit;
    if (!__syncthreads_and(tid == 0 && have ? mbar_wait(bars + u % kHalfStages, (unsigned)((u / kHalfStages) & 1))
                                            : true)) {
      ok = false;
      break;
    }
    if (tid == 0 && u >= 1 && issued < nunit) {
      fence_proxy_async();  // the generic reads of unit u-1's stage before its refill
      issue(issued);
      ++issued;
    }
    // the previous tile's column table (written after its second half) is complete
    if ((u & 1) == 0 && u >= 2 && prevIJ.x != prevIJ.y) sym_columns_out(colred, prevIJ, prevI, nb, lane, wid, tp);
    if (!have) break;
    const int s = u % kHalfStages, h = u & 1;
    const int2 IJ = stile[s];
    const int Il = lblk ? lblk[IJ.x] : IJ.x, Jl = lblk ? lblk[IJ.y] : IJ.y;  // slot blocks
    prevIJ = IJ;
    prevI = Il;
    const bool diag = IJ.x == IJ.y;
    const float4 *__restrict__ T = (const float4 *)(ssm + (size_t)s * kHalfStageBytes);
    const float2 *__restrict__ fr = (const float2 *)(ssm + (size_t)s * kHalfStageBytes + kHalfTileBytes);
    const float2 *__restrict__ fc = fr + HR;
    float2 fcol[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) fcol[j] = fc[tj + 16 * j];
    float rA[R][2], rC[R][2];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int row = ti * R + i;
      const float2 fs = fr[row];
      float4 e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) e[j] = T[row * kTile + tj + 16 * j];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j == 0) {
          ff_prod(rA[i][0], rA[i][1], fcol[j], e[j].x, e[j].y);
          ff_prod(rC[i][0], rC[i][1], fcol[j], e[j].z, e[j].w);
        } else {
          ff_mac_lazy(rA[i][0], rA[i][1], fcol[j], e[j].x, e[j].y);
          ff_mac_lazy(rC[i][0], rC[i][1], fcol[j], e[j].z, e[j].w);
        }
        if (!diag) {
          if (h == 0 && i == 0) {
            ff_prod(cA[j][0], cA[j][1], fs, e[j].z, e[j].w);
            ff_prod(cC[j][0], cC[j][1], fs, e[j].x, e[j].y);
          } else {
            ff_mac_lazy(cA[j][0], cA[j][1], fs, e[j].z, e[j].w);
            ff_mac_lazy(cC[j][0], cC[j][1], fs, e[j].x, e[j].y);
          }
        }
      }
    }
    // rows: the 16 lanes of a half-warp share them; lanes 4m .. 4m + 3 end with value m = (row, A | C)
    {
      float2 v[NV];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        v[2 * i] = make_float2(rA[i][0], rA[i][1]);
        v[2 * i + 1] = make_float2(rC[i][0], rC[i][1]);
      }
      ff_reduce_scatter<NV, 8>(v, lane);
      const int idx = tj >> 2;
      if ((tj & 3) == 0) {
        const int row = IJ.x * kTile + h * HR + ti * R + (idx >> 1);
        ((float2 *)tp)[2 * ((long long)row * nb + Jl) + (idx & 1)] = v[0];
      }
    }
    if (!diag && h == 1) {
      // columns of the whole tile: lanes tj and tj + 16 share them (one level), then the warps
      // (after the next unit's barrier)
      const bool up = lane & 16;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int jk = m >> 1, jo = jk + 2;  // kept / sent column slot
        const float2 a = (m & 1) ? make_float2(cC[jk][0], cC[jk][1]) : make_float2(cA[jk][0], cA[jk][1]);
        const float2 c = (m & 1) ? make_float2(cC[jo][0], cC[jo][1]) : make_float2(cA[jo][0], cA[jo][1]);
        const float2 send = up ? a : c, keep = up ? c : a;
        const float2 w = ff_add(keep, make_float2(__shfl_xor_sync(0xFFFFFFFFu, send.x, 16),
                                                  __shfl_xor_sync(0xFFFFFFFFu, send.y, 16)));
        const int col = tj + 16 * ((up ? 2 : 0) + jk);
        colred[(wid * 2 + (m & 1)) * kTile + col] = w;
      }
    }
  }
  if (!ok) {
    *err = 2;
    if (tid == 0) {  // drain: wait (bounded) for every copy this CTA issued
      for (int k = 0; k < kHalfStages; ++k) {
        const int uses = issued / kHalfStages + (k < issued % kHalfStages ? 1 : 0);
        if (uses > 0) mbar_wait(bars + k, (unsigned)((uses - 1) & 1));
      }
    }
  }
}

// ------------------------------------------------------------ finalisers

// Row totals of the (A, B) partials (coefficient variants) or of the literal sums.
__device__ __forceinline__ void row_partials(const int *__restrict__ item_ptr, const Part4 *__restrict__ part, int r,
                                             double &A, double &B) {
  A = 0.0;
  B = 0.0;
  for (int i = item_ptr[r]; i < item_ptr[r + 1]; ++i) {
    const Part4 v = part[i];
    A += v.x;
    B += v.y;
  }
}

// Where a row's partial sums (A, B) come from: the work items of its row (one Part4 each)
// or, for the symmetric tile sweep, one double2 per block of partner states.
struct ItemSrc {
  const int *item_ptr;
  const Part4 *part;
  __device__ __forceinline__ void get(int r, double &A, double &B) const { row_partials(item_ptr, part, r, A, B); }
};
struct TileSrc {
  const float4 *tp;  // [nsp][nb]: state-major, one partial (A hi, A lo, C hi, C lo) per block of partner states
  int nb, nsp;
  // batched tiles: the padded row of every state and the block table (the number of partner
  // blocks of a state is its system's, binfo[block].w); null for one system
  const int *pmap = nullptr;
  const int4 *binfo = nullptr;
};

// Collision epilogue fused with the RK4 stage arithmetic.
//   STAGE < 0 : out[r] = I_r (plain pb_collision)
//   STAGE 0..3: classic RK4 stage k_{STAGE+1} = I[y]; see the host driver for buffers.
// The per-state inputs of the epilogue, loaded before the partial sums so that their latency
// overlaps the partials' (the epilogues are a chain of dependent loads otherwise).
struct FinIn {
  double R, y, f, acc;
};
template <bool LIT, int STAGE>
__device__ __forceinline__ FinIn fin_load(int r, const double *__restrict__ R, const double *__restrict__ ysrc,
                                          const double *__restrict__ f, const double *__restrict__ acc) {
  FinIn v{0.0, 0.0, 0.0, 0.0};
  if (!LIT) {
    v.R = R[r];
    v.y = ysrc[r];
  }
  if (STAGE >= 0) v.f = f[r];
  if (STAGE >= 1) v.acc = acc[r];
  return v;
}

// out[r] = I (STAGE < 0), or the RK4 stage arithmetic with k_{STAGE+1} = I
// ry: the state's row of yff when that is a padded state space (batched tiles), else r
template <int STAGE, bool GSTATE>
__device__ __forceinline__ void fin_stage(int r, double I, const FinIn &in, double *__restrict__ out,
                                          double *__restrict__ f, double *__restrict__ acc, double *__restrict__ y,
                                          float2 *__restrict__ yff, double dt, int ry = -1) {
  if (STAGE < 0) {
    out[r] = I;
    return;
  }
  const double fr = in.f;
  double yn;
  if (STAGE == 0) {
    acc[r] = I;
    yn = fr + 0.5 * dt * I;
  } else if (STAGE == 1) {
    acc[r] = in.acc + 2.0 * I;
    yn = fr + 0.5 * dt * I;
  } else if (STAGE == 2) {
    acc[r] = in.acc + 2.0 * I;
    yn = fr + dt * I;
  } else {
    yn = fr + dt / 6.0 * (in.acc + I);
    f[r] = yn;
  }
  y[r] = yn;
  if (GSTATE)
    rec_set_f(reinterpret_cast<uint4 *>(yff) + r, yn);  // yff points at the uint4 record array
  else
    yff[ry < 0 ? r : ry] = ff_split(yn);
}

template <bool LIT, int STAGE, bool GSTATE>
__device__ __forceinline__ void fin_apply(int r, double A, double B, double c, const FinIn &in,
                                          double *__restrict__ out, double *__restrict__ f, double *__restrict__ acc,
                                          double *__restrict__ y, float2 *__restrict__ yff, double dt, int ry = -1) {
  fin_stage<STAGE, GSTATE>(r, LIT ? -c * A : c * (A - in.y * (in.R - B)), in, out, f, acc, y, yff, dt, ry);
}

template <bool LIT, int STAGE, bool GSTATE = false, typename SRC = ItemSrc>
__global__ void k_fin_coll(SRC src, int ns, double c, const double *__restrict__ R, const double *__restrict__ ysrc,
                           double *__restrict__ out, double *__restrict__ f, double *__restrict__ acc,
                           double *__restrict__ y, float2 *__restrict__ yff, double dt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ns) return;
  const FinIn in = fin_load<LIT, STAGE>(r, R, ysrc, f, acc);
  double A, B;
  src.get(r, A, B);
  fin_apply<LIT, STAGE, GSTATE>(r, A, B, c, in, out, f, acc, y, yff, dt);
}

// The same epilogue over symmetric-tile partials, one warp per state: lanes add the block
// partials k = lane, lane + 32, ... and a fixed shuffle tree combines them, all in float-float
// (FP64 adds run at 1/64 of the FP32 rate on this part: 75 double partials per state and a
// double shuffle tree made this epilogue cost as much as a fifth of the sweep).  RATE: 1/tau.
// The epilogue of the symmetric tile sweep: a 256-thread CTA takes 32 states.  Each warp adds
// the block partials of 4 states (lanes over the blocks, then one 32-lane float-float
// reduce-scatter of the 8 values) into a shared table; warp 0 then applies Eq. 2 and the RK4
// stage arithmetic in FP64 to the 32 states at once, one lane per state (FP64 instructions
// cost the same with one active lane as with 32 on this part, so a lane-0-per-state epilogue
// spent most of its time there).  RATE: 1/tau.
// SPC states per CTA (8 or 32; few states take 8, for more CTAs in flight)
template <int STAGE, bool RATE = false, int SPC = 32>
__global__ void __launch_bounds__(256) k_fin_tiles(TileSrc src, int ns, double c, const double *__restrict__ R,
                                                   const double *__restrict__ ysrc, double *__restrict__ out,
                                                   double *__restrict__ f, double *__restrict__ acc,
                                                   double *__restrict__ y, float2 *__restrict__ yff, double dt) {
  constexpr int SPW = SPC / 8, NV = 2 * SPW, LPV = 32 / NV;  // states per warp, values, lanes per value
  __shared__ float4 tot[SPC];  // (A hi, A lo, C hi, C lo) per state
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int base = blockIdx.x * SPC;
  // warp 0 loads its state's epilogue inputs first, so that their latency overlaps the partials'
  const int r0 = base + lane;
  FinIn in{0.0, 0.0, 0.0, 0.0};
  if (wid == 0 && lane < SPC && r0 < ns) {
    if (RATE) in.R = R[r0];
    else in = fin_load<false, STAGE>(r0, R, ysrc, f, acc);
  }
  // partials are stored for every padded state (r < nsp); the first three of every lane for
  // the warp's states are loaded together (up to 96 partner blocks), the rest after
  const int nb = src.nb;
  float4 w[SPW][3];
  int nbq[SPW];  // partner blocks of each state
#pragma unroll
  for (int q = 0; q < SPW; ++q) {
    const int r = base + SPW * wid + q;
    const int pr = src.pmap && r < src.nsp ? src.pmap[r] : r;
    nbq[q] = src.binfo && r < src.nsp ? src.binfo[pr / kTile].w : nb;
    const float4 *__restrict__ row = src.tp + (long long)pr * nb;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int k = lane + 32 * m;
      w[q][m] = r < src.nsp && k < nbq[q] ? row[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  float2 v[NV];
#pragma unroll
  for (int q = 0; q < SPW; ++q) {
    v[2 * q] = make_float2(w[q][0].x, w[q][0].y);
    v[2 * q + 1] = make_float2(w[q][0].z, w[q][0].w);
#pragma unroll
    for (int m = 1; m < 3; ++m) {
      v[2 * q] = ff_add(v[2 * q], make_float2(w[q][m].x, w[q][m].y));
      v[2 * q + 1] = ff_add(v[2 * q + 1], make_float2(w[q][m].z, w[q][m].w));
    }
    const int r = base + SPW * wid + q;
    if (r < src.nsp) {
      const float4 *__restrict__ row = src.tp + (long long)(src.pmap ? src.pmap[r] : r) * nb;
      for (int k = lane + 96; k < nbq[q]; k += 32) {
        const float4 x = row[k];
        v[2 * q] = ff_add(v[2 * q], make_float2(x.x, x.y));
        v[2 * q + 1] = ff_add(v[2 * q + 1], make_float2(x.z, x.w));
      }
    }
  }
  ff_reduce_scatter<NV, 16>(v, lane);
  if ((lane & (LPV - 1)) == 0) {
    const int idx = lane / LPV;  // the top lane bits: (state q, A | C)
    float *t = reinterpret_cast<float *>(tot + SPW * wid + (idx >> 1)) + 2 * (idx & 1);
    t[0] = v[0].x;
    t[1] = v[0].y;
  }
  __syncthreads();
  if (wid != 0 || lane >= SPC || r0 >= ns) return;
  const float4 T = tot[lane];
  const double A = ff_to_double(T.x, T.y), B = ff_to_double(T.z, T.w) - A;
  if (RATE)
    out[r0] = c * (in.R - B);
  else
    fin_apply<false, STAGE, false>(r0, A, B, c, in, out, f, acc, y, yff, dt, src.pmap ? src.pmap[r0] : r0);
}

template <bool LIT, typename SRC = ItemSrc>
__global__ void k_fin_rate(SRC src, int ns, double c, const double *__restrict__ R, double *__restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ns) return;
  const double Rr = LIT ? 0.0 : R[r];
  double A, B;
  src.get(r, A, B);
  out[r] = LIT ? c * A : c * (Rr - B);
}

// F_new = tau (v + sum W F); ff copy for the next pass; per-block max |dF| and max |F|.
// max over the block of (a, b), both non-negative: warp shuffles, then one step through shared
// memory (exact, so the order does not matter); the result is valid in thread 0
__device__ __forceinline__ double2 block_max2(double a, double b) {
  __shared__ double2 wm[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xFFFFFFFFu, a, o));
    b = fmax(b, __shfl_xor_sync(0xFFFFFFFFu, b, o));
  }
  if (lane == 0) wm[wid] = make_double2(a, b);
  __syncthreads();
  double2 v = make_double2(0.0, 0.0);
  if (wid == 0) {
    v = lane < (int)((blockDim.x + 31) >> 5) ? wm[lane] : make_double2(0.0, 0.0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x = fmax(v.x, __shfl_xor_sync(0xFFFFFFFFu, v.x, o));
      v.y = fmax(v.y, __shfl_xor_sync(0xFFFFFFFFu, v.y, o));
    }
  }
  return v;
}

__global__ void __launch_bounds__(256) k_fin_tr(const int *__restrict__ item_ptr, const Part4 *__restrict__ part,
                                                int ns, const double *__restrict__ tau,
                                                const double *__restrict__ vel3, const double *__restrict__ Fold,
                                                double *__restrict__ Fnew, float2 *__restrict__ Fff,
                                                double2 *__restrict__ red) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double dm = 0.0, fm = 0.0;
  if (r < ns) {
    // the row's own inputs first, so that their latency overlaps that of the partials
    const double t = tau[r];
    double vv[3], fo[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      vv[a] = vel3[3 * r + a];
      fo[a] = Fold ? Fold[3 * r + a] : 0.0;
    }
    double X = 0.0, Y = 0.0, Z = 0.0;
    const int i1 = item_ptr[r + 1];
    for (int i = item_ptr[r]; i < i1; ++i) {
      const Part4 v = part[i];
      X += v.x;
      Y += v.y;
      Z += v.z;
    }
    const double S[3] = {X, Y, Z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double Fn = t * (vv[a] + S[a]);
      if (Fold) dm = fmax(dm, fabs(Fn - fo[a]));
      fm = fmax(fm, fabs(Fn));
      Fnew[3 * r + a] = Fn;
      Fff[3 * r + a] = ff_split(Fn);
    }
  }
  const double2 m = block_max2(dm, fm);
  if (threadIdx.x == 0) red[blockIdx.x] = m;
}

__global__ void k_red_final(const double2 *__restrict__ red, int n, double *__restrict__ out) {
  double d = 0.0, m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d = fmax(d, red[i].x);
    m = fmax(m, red[i].y);
  }
  const double2 v = block_max2(d, m);
  if (threadIdx.x == 0) {
    out[0] = v.y > 0.0 ? v.x / v.y : 0.0;
    out[1] = v.x;
    out[2] = v.y;
  }
}

// F^0 = tau v and its float-float copy
__global__ void k_tr_init(const double *__restrict__ tau, const double *__restrict__ vel3, int ns,
                          double *__restrict__ F, float2 *__restrict__ Fff) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * ns) return;
  const double v = tau[i / 3] * vel3[i];
  F[i] = v;
  Fff[i] = ff_split(v);
}

// Deterministic single-block sums: out[0] = sum f, out[1] = sum eps f, out[2] = sum I.
__global__ void k_observables(const double *__restrict__ f, const double *__restrict__ eps,
                              const double *__restrict__ I, int ns, double *__restrict__ out) {
  __shared__ double s0[1024], s1[1024], s2[1024];
  double a = 0.0, b = 0.0, d = 0.0;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    a += f[i];
    b += eps[i] * f[i];
    d += I[i];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  s2[threadIdx.x] = d;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
    out[2] = s2[0];
  }
}

}  // namespace dev
}  // namespace pb
