// FP32 coefficient tiles (PB_VARIANT_C32): the collision sweep of Eq. 2 over the upper block
// triangle of the branch-merged pair matrix, stored as 64 x 64 tiles of FP32 (P_in, P_out),
// 8 bytes per state pair: half the bytes of the float-float tiles.  Included by device.cu after
// kernels.cuh (it uses the tile, mbarrier and bulk-copy helpers there).
//
// Why a per-entry net term.  The pair (s, p) adds
//     n(s,p) = P_in f_p (1 - f_s) - P_out f_s (1 - f_p)
// to I_s / c and -n(s,p) to I_p / c (the reverse channel swaps P_in and P_out).  Near a steady
// state the two products are much larger than their difference, so sums of them (the A and C
// sums of the float-float sweep) rounded to FP32 carry errors of 2^-24 of the gross scattering,
// which the closing difference turns into 1e-6 of df/dt and more along a 1000-step trajectory.
// Here every entry forms n(s,p) itself, with the larger product made exact by an FMA error term:
//     n = P_in f_p - P_out f_s - d f_s f_p,   d = P_in - P_out,
//     u = fl(P_in f_p),  e = P_in f_p - u (exact, one FMA),  v = fl(P_out f_s - u) (one FMA),
//     n = fl(-d fl(f_s f_p) + (e - v)),
// so the rounding left in n is relative to n.  The occupations are float-float (f = f_h + f_l);
// n is taken at f_h and the entry adds its first-order change in f_l,
//     t(s,p) = n + f_l,p (P_in - f_s d) - f_l,s (P_out + f_p d)
// (dn/df_p = P_in - f_s d, dn/df_s = -(P_out + f_p d); the second-order term f_l,s f_l,p d is
// below 2^-48 of the products).  t(p,s) = -t(s,p) for every f, so the row of s adds t and the
// row of p subtracts the same FP32 value: each state needs one sum, I_s = c sum_p t(s,p).
//
namespace pb {
namespace dev {

constexpr int kC32Threads = 256;
constexpr int kC32RatioUlps = 2;
constexpr unsigned kC32TileBytes = kTile * kTile * sizeof(float2);
constexpr unsigned kC32StageBytes = kC32TileBytes + 2 * kTile * sizeof(float2);
constexpr size_t kC32ColFloats = (size_t)(kC32Threads / 32) * kTile;  // [8 warps][64 columns]
// dynamic shared memory of a launch shape with NST stages (and the double-buffered column table)
template <int NST>
constexpr size_t c32_smem() {
  return (size_t)NST * kC32StageBytes + 128 + 2 * kC32ColFloats * sizeof(float);
}

// (a, b) ~ (P_in, P_out) in FP32 with the ratio kept (see above); zero stays zero.
__device__ __forceinline__ float2 c32_round_pair(double pin, double pout) {
  const float a0 = __double2float_rn(pin);
  if (!(a0 > 0.f) || !(pout > 0.0)) return make_float2(a0, __double2float_rn(pout));
  const double r = pout / pin;
  float ba = a0, bb = __double2float_rn((double)a0 * r);
  double be = fabs((double)bb / (double)ba - r);
  for (int k = -kC32RatioUlps; k <= kC32RatioUlps; ++k) {
    if (k == 0) continue;
    const float a = __int_as_float(__float_as_int(a0) + k);
    if (!(a > 0.f) || isinf(a)) continue;
    const float b = __double2float_rn((double)a * r);
    if (!(b > 0.f) || isinf(b)) continue;
    const double e = fabs((double)b / (double)a - r);
    if (e < be) {
      be = e;
      ba = a;
      bb = b;
    }
  }
  return make_float2(ba, bb);
}

// tc[t][i][j] = rounded (P_in, P_out) of pair (64 I + i, 64 J + j) from the branch-merged
// float-float coefficients of complete rows (entry (s, p) of row s is at srp[s] + p); zero
// outside the nstate states.
__global__ void k_tiles_fill_c32(const int2 *__restrict__ tiles, int nt, const float2 *__restrict__ coefA,
                                 const float2 *__restrict__ coefB, const long long *__restrict__ srp, int ns,
                                 float2 *__restrict__ tc) {
  const long long n = (long long)nt * kTile * kTile;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / (kTile * kTile)), k = (int)(e % (kTile * kTile));
    const int2 IJ = tiles[t];
    const int s = IJ.x * kTile + k / kTile, p = IJ.y * kTile + k % kTile;
    float2 v = make_float2(0.f, 0.f);
    if (s < ns && p < ns) {
      const long long c = srp[s] + p;
      const float2 a = coefA[c], b = coefB[c];
      const double pin = ff_to_double(a.x, a.y), pout = pin + ff_to_double(b.x, b.y);
      v = c32_round_pair(pin, pout);
    }
    tc[e] = v;
  }
}

// The symmetric tiles from branch-merged pair rows that need not be complete (the batch's
// systems, or one system whose rows miss some partners): one warp per row s, every stored pair
// (s, p) whose block pair (I, J) lies in the upper triangle (I <= J) written to its tile entry;
// the tiles were zeroed before, pairs without channels stay zero, and zero padding entries are
// skipped.  Several systems share one padded block space through pmap (each state's padded row)
// and binfo[g] of block g = (first block of its system, the system's first tile, its states, its
// blocks); with both null there is one system of ns states in nbs blocks.  Tiles are numbered
// row-major over each system's upper block triangle.  C32: the pairs rounded to FP32 with their
// ratio kept, else float-float (float4 per entry).
template <bool C32, typename IDX>
__global__ void k_tiles_scatter(const long long *__restrict__ srp, int ns, const IDX *__restrict__ pidx,
                                const float2 *__restrict__ coefA, const float2 *__restrict__ coefB,
                                const int *__restrict__ pmap, const int4 *__restrict__ binfo, int nbs,
                                void *__restrict__ tc) {
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)(((long long)gridDim.x * blockDim.x) >> 5);
  for (int r = w0; r < ns; r += nw) {
    const int pr = pmap ? pmap[r] : r;
    const int4 bi = binfo ? binfo[pr / kTile] : make_int4(0, 0, ns, nbs);
    const int I = pr / kTile - bi.x;
    for (long long e = srp[r] + lane; e < srp[r + 1]; e += 32) {
      const float2 a = coefA[e], b = coefB[e];
      if (a.x == 0.f && a.y == 0.f && b.x == 0.f && b.y == 0.f) continue;
      const int pp = pmap ? pmap[pidx[e]] : (int)pidx[e];
      const int J = pp / kTile - bi.x;
      if (J < I) continue;
      const long long t = (long long)bi.y + (long long)I * (2 * bi.w - I + 1) / 2 + (J - I);
      const long long k = t * kTile * kTile + (pr % kTile) * kTile + pp % kTile;
      const double pin = ff_to_double(a.x, a.y), pout = pin + ff_to_double(b.x, b.y);
      if (C32) {
        ((float2 *)tc)[k] = c32_round_pair(pin, pout);
      } else {
        const float2 x = ff_split(pin), y = ff_split(pout);
        ((float4 *)tc)[k] = make_float4(x.x, x.y, y.x, y.y);
      }
    }
  }
}

// t(s, p) above from the entry's rounded (P_in, P_out) = (a, b) and the float-float occupations
// fs of s and fp of p
__device__ __forceinline__ float c32_term(float a, float b, float2 fs, float2 fp) {
  const float d = __fsub_rn(a, b);
  const float u = __fmul_rn(a, fp.x);
  const float ex = __fmaf_rn(a, fp.x, -u);
  const float v = __fmaf_rn(b, fs.x, -u);
  const float w = __fmul_rn(fs.x, fp.x);
  float t = __fmaf_rn(-d, w, __fsub_rn(ex, v));
  t = __fmaf_rn(fp.y, __fmaf_rn(-fs.x, d, a), t);
  return __fmaf_rn(-fs.y, __fmaf_rn(fp.x, d, b), t);
}

// reduce-scatter of NV floats over the 2 * TOP lanes that differ in lane bits log2 TOP .. 0: at
// the end v[0] holds the total of value index idx(lane) = those bits of the lane, most
// significant first (the float-float version is ff_reduce_scatter)
template <int NV, int TOP>
__device__ __forceinline__ void f32_reduce_scatter(float (&v)[NV], int lane) {
  int n = NV;
#pragma unroll
  for (int mask = TOP; mask > 0; mask >>= 1) {
    if (n > 1) {
      const bool up = lane & mask;
      const int h = n >> 1;
#pragma unroll
      for (int k = 0; k < NV / 2; ++k) {
        if (k < h) {
          const float send = up ? v[k] : v[k + h], keep = up ? v[k + h] : v[k];
          v[k] = __fadd_rn(keep, __shfl_xor_sync(0xFFFFFFFFu, send, mask));
        }
      }
      n = h;
    } else {
      v[0] = __fadd_rn(v[0], __shfl_xor_sync(0xFFFFFFFFu, v[0], mask));
    }
  }
}

// the column sums of a finished off-diagonal tile: threads 0..63 add the 8 warps' values of
// one column each and write them to the column state's partial for the tile's row block (slot
// slotI)
__device__ __forceinline__ void c32_columns_out(const float *__restrict__ colred, int2 IJ, int slotI, int nb, int tid,
                                                float *__restrict__ tp) {
  if (tid >= kTile) return;
  float acc = colred[tid];
#pragma unroll
  for (int w = 1; w < kC32Threads / 32; ++w) acc = __fadd_rn(acc, colred[w * kTile + tid]);
  tp[(long long)(IJ.y * kTile + tid) * nb + slotI] = acc;
}

// One persistent 256-thread CTA (CPS per SM) streams its share of the tiles through NST
// shared-memory stages filled by bulk copies (thread 0 issues, completion counted in bytes on
// one mbarrier per stage, every wait bounded), as k_stream_sym_bulk does for the float-float
// tiles.  Thread (ti, tj) takes rows 4 ti .. 4 ti + 3 and columns tj + 16 j.  One FP32 partial
// per (state, block of partner states): MODE_COLL the sum of t above; MODE_RATE the sum of the
// 1/tau_s summands P_out + f_p d (row s) and P_in - f_s d (column p, the reverse channel), each
// with its f_l term.  The per-warp column table is double buffered and combined in the next
// iteration, so a tile costs one CTA barrier.
// lblk (batched sweep, else null): the block index of each block within its instance, which
// numbers the partial slots.  rev: take the tile list from its end (tile nt - 1 - t in place of
// t), so that a sweep following one in list order starts on the tiles the L2 still holds.
template <int MODE, int NST, int CPS>
__global__ void __launch_bounds__(kC32Threads, CPS) k_stream_c32(const int2 *__restrict__ tiles, int nt,
                                                                  const float2 *__restrict__ tc,
                                                                  const float2 *__restrict__ fg, int ns, int nb,
                                                                  float *__restrict__ tp, int *__restrict__ err,
                                                                  const int *__restrict__ lblk = nullptr,
                                                                  int rev = 0) {
  // the stage of tile k - 1 is refilled (with tile k - 1 + NST) only after the wait for tile k, so
  // one stage would wait for a copy not yet issued
  static_assert(NST >= 2 && NST <= 8, "the ring needs 2..8 stages");
  constexpr int R = 4;
  extern __shared__ __align__(128) unsigned char ssm[];
  unsigned long long *bars = (unsigned long long *)(ssm + NST * kC32StageBytes);
  int2 *stile = (int2 *)(bars + NST);
  float *colred0 = (float *)(ssm + NST * kC32StageBytes + 128);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, tj = tid & 15, ti = tid >> 4;
  const int G = (int)gridDim.x;
  const int nloc = (int)blockIdx.x < nt ? (nt - 1 - (int)blockIdx.x) / G + 1 : 0;
  for (int i = tid; i < NST * 2 * kTile; i += kC32Threads) {
    float2 *fz = (float2 *)(ssm + (i / (2 * kTile)) * kC32StageBytes + kC32TileBytes);
    fz[i % (2 * kTile)] = make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    for (int k = 0; k < NST; ++k) mbar_init(bars + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  __syncthreads();
  int issued = 0;
  auto tix = [&](int k) {  // the CTA's k-th tile
    const int t = (int)blockIdx.x + k * G;
    return rev ? nt - 1 - t : t;
  };
  auto issue = [&](int k, int2 IJ) {
    const int s = k % NST;
    const int t = tix(k);
    stile[s] = IJ;
    unsigned char *buf = ssm + (size_t)s * kC32StageBytes;
    const int nr = min(kTile, ns - IJ.x * kTile), nc = min(kTile, ns - IJ.y * kTile);
    const unsigned br = (unsigned)(nr * sizeof(float2) + 15) / 16 * 16, bc = (unsigned)(nc * sizeof(float2) + 15) / 16 * 16;
    mbar_expect_tx(bars + s, kC32TileBytes + br + bc);
    const unsigned char *src = (const unsigned char *)(tc + (size_t)t * kTile * kTile);
#pragma unroll
    for (int q = 0; q < 2; ++q) bulk_g2s(buf + q * (kC32TileBytes / 2), src + q * (kC32TileBytes / 2), kC32TileBytes / 2, bars + s);
    bulk_g2s(buf + kC32TileBytes, fg + (size_t)IJ.x * kTile, br, bars + s);
    bulk_g2s(buf + kC32TileBytes + kTile * sizeof(float2), fg + (size_t)IJ.y * kTile, bc, bars + s);
  };
  if (tid == 0)
    for (; issued < NST && issued < nloc; ++issued) issue(issued, tiles[tix(issued)]);
  int2 nextIJ = make_int2(0, 0);
  if (tid == 0 && issued < nloc) nextIJ = tiles[tix(issued)];
  int2 prevIJ = make_int2(0, 0);
  int prevI = 0;
  bool ok = true;
  for (int k = 0; k <= nloc; ++k) {
    const bool have = k < nloc;
    if (!__syncthreads_and(tid == 0 && have ? mbar_wait(bars + k % NST, (unsigned)((k / NST) & 1)) : true)) {
      ok = false;
      break;
    }
    if (tid == 0 && k >= 1 && issued < nloc) {
      fence_proxy_async();  // the generic reads of tile k-1's stage before its refill
      issue(issued, nextIJ);
      ++issued;
      if (issued < nloc) nextIJ = tiles[tix(issued)];
    }
    if (k >= 1 && prevIJ.x != prevIJ.y)
      c32_columns_out(colred0 + ((k - 1) & 1) * kC32ColFloats, prevIJ, prevI, nb, tid, tp);
    if (!have) break;
    const int s = k % NST;
    const int2 IJ = stile[s];
    const int Il = lblk ? lblk[IJ.x] : IJ.x, Jl = lblk ? lblk[IJ.y] : IJ.y;  // slot blocks
    prevIJ = IJ;
    prevI = Il;
    const bool diag = IJ.x == IJ.y;
    const float2 *__restrict__ T = (const float2 *)(ssm + (size_t)s * kC32StageBytes);
    const float2 *__restrict__ fr = (const float2 *)(ssm + (size_t)s * kC32StageBytes + kC32TileBytes);
    const float2 *__restrict__ fc = fr + kTile;
    float2 fcol[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) fcol[j] = fc[tj + 16 * j];
    float rv[R], cv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) rv[i] = cv[i] = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int row = ti * R + i;
      const float2 fs = fr[row];
      float2 e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) e[j] = T[row * kTile + tj + 16 * j];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float a = e[j].x, b = e[j].y, fp = fcol[j].x, flp = fcol[j].y;
        if (MODE == MODE_COLL) {
          const float t = c32_term(a, b, fs, fcol[j]);
          rv[i] = __fadd_rn(rv[i], t);
          if (!diag) cv[j] = __fsub_rn(cv[j], t);
        } else {  // 1/tau summands: row s: P_out + f_p d; column p (reverse channel): P_in - f_s d
          const float d = __fsub_rn(a, b);
          rv[i] = __fadd_rn(rv[i], __fmaf_rn(flp, d, __fmaf_rn(fp, d, b)));
          if (!diag) cv[j] = __fadd_rn(cv[j], __fmaf_rn(-fs.y, d, __fmaf_rn(-fs.x, d, a)));
        }
      }
    }
    // rows: the 16 lanes of a half-warp share them; lanes 4i .. 4i + 3 end with the total of row i
    f32_reduce_scatter<R, 8>(rv, lane);
    if ((tj & 3) == 0) tp[(long long)(IJ.x * kTile + ti * R + (tj >> 2)) * nb + Jl] = rv[0];
    if (!diag) {
      // columns: lanes tj and tj + 16 share them (one level), then the 8 warps (next iteration)
      float *colred = colred0 + (k & 1) * kC32ColFloats;
      const bool up = lane & 16;
#pragma unroll
      for (int jk = 0; jk < 2; ++jk) {
        const int jo = jk + 2;  // kept / sent column slot
        const float kept = up ? cv[jo] : cv[jk], sent = up ? cv[jk] : cv[jo];
        colred[wid * kTile + tj + 16 * ((up ? 2 : 0) + jk)] = __fadd_rn(kept, __shfl_xor_sync(0xFFFFFFFFu, sent, 16));
      }
    }
  }
  if (!ok) {
    *err = 2;
    if (tid == 0) {
      for (int k = 0; k < NST; ++k) {
        const int uses = issued / NST + (k < issued % NST ? 1 : 0);
        if (uses > 0) mbar_wait(bars + k, (unsigned)((uses - 1) & 1));
      }
    }
  }
}

// The same sweep in half-tiles (32 rows x 64 columns, 16 KB, contiguous in the tile): a tile's
// column sums stay in registers across its two halves and go through the per-warp table after the
// second, which is combined after the next unit's barrier (columns are written only every other
// unit, so one table suffices).  Three 17 KB stages and the 2 KB table take 53 KB, so four CTAs
// (32 warps) fit on an SM.  Thread (ti, tj) takes rows 2 ti, 2 ti + 1 of the unit and columns
// tj + 16 j.
constexpr unsigned kC32HalfBytes = kC32TileBytes / 2;
constexpr unsigned kC32HalfStageBytes = kC32HalfBytes + (kTile / 2 + kTile) * sizeof(float2);
template <int NST>
constexpr size_t c32_half_smem() {
  return (size_t)NST * kC32HalfStageBytes + 128 + kC32ColFloats * sizeof(float);
}

template <int MODE, int NST, int CPS>
__global__ void __launch_bounds__(kC32Threads, CPS) k_stream_c32_half(const int2 *__restrict__ tiles, int nt,
                                                                       const float2 *__restrict__ tc,
                                                                       const float2 *__restrict__ fg, int ns, int nb,
                                                                       float *__restrict__ tp, int *__restrict__ err,
                                                                       const int *__restrict__ lblk = nullptr,
                                                                       int rev = 0) {
  static_assert(NST >= 2 && NST <= 8, "the ring needs 2..8 stages");
  constexpr int R = 2, HR = kTile / 2;
  extern __shared__ __align__(128) unsigned char ssm[];
  unsigned long long *bars = (unsigned long long *)(ssm + NST * kC32HalfStageBytes);
  int2 *stile = (int2 *)(bars + NST);
  float *colred = (float *)(ssm + NST * kC32HalfStageBytes + 128);  // [8 warps][64 columns]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, tj = tid & 15, ti = tid >> 4;
  const int G = (int)gridDim.x;
  const int nloc = (int)blockIdx.x < nt ? (nt - 1 - (int)blockIdx.x) / G + 1 : 0;
  const int nunit = 2 * nloc;
  for (int i = tid; i < NST * (HR + kTile); i += kC32Threads) {
    float2 *fz = (float2 *)(ssm + (i / (HR + kTile)) * kC32HalfStageBytes + kC32HalfBytes);
    fz[i % (HR + kTile)] = make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    for (int k = 0; k < NST; ++k) mbar_init(bars + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  __syncthreads();
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
    const int k = v >> 1, h = v & 1, s = v % NST;
    if (h == 0 && k > 0) {
      issIJ = aheadIJ;
      if (k + 1 < nloc) aheadIJ = tiles[tix(k + 1)];
    }
    const int t = tix(k);
    stile[s] = issIJ;
    unsigned char *buf = ssm + (size_t)s * kC32HalfStageBytes;
    const int nr = min(HR, ns - (issIJ.x * kTile + h * HR)), nc = min(kTile, ns - issIJ.y * kTile);
    const unsigned br = nr > 0 ? (unsigned)(nr * sizeof(float2) + 15) / 16 * 16 : 0u;
    const unsigned bc = (unsigned)(nc * sizeof(float2) + 15) / 16 * 16;
    mbar_expect_tx(bars + s, kC32HalfBytes + br + bc);
    const unsigned char *src = (const unsigned char *)(tc + (size_t)t * kTile * kTile) + (size_t)h * kC32HalfBytes;
    bulk_g2s(buf, src, kC32HalfBytes, bars + s);
    if (br) bulk_g2s(buf + kC32HalfBytes, fg + (size_t)issIJ.x * kTile + h * HR, br, bars + s);
    bulk_g2s(buf + kC32HalfBytes + HR * sizeof(float2), fg + (size_t)issIJ.y * kTile, bc, bars + s);
  };
  if (tid == 0)
    for (; issued < NST && issued < nunit; ++issued) issue(issued);
  int2 prevIJ = make_int2(0, 0);
  int prevI = 0;
  bool ok = true;
  float cv[4];  // column sums of the current tile, carried across its halves
  for (int u = 0; u <= nunit; ++u) {
    const bool have = u < nunit;
    if (!__syncthreads_and(tid == 0 && have ? mbar_wait(bars + u % NST, (unsigned)((u / NST) & 1)) : true)) {
      ok = false;
      break;
    }
    if (tid == 0 && u >= 1 && issued < nunit) {
      fence_proxy_async();  // the generic reads of unit u-1's stage before its refill
      issue(issued);
      ++issued;
    }
    if ((u & 1) == 0 && u >= 2 && prevIJ.x != prevIJ.y) c32_columns_out(colred, prevIJ, prevI, nb, tid, tp);
    if (!have) break;
    const int s = u % NST, h = u & 1;
    const int2 IJ = stile[s];
    const int Il = lblk ? lblk[IJ.x] : IJ.x, Jl = lblk ? lblk[IJ.y] : IJ.y;  // slot blocks
    prevIJ = IJ;
    prevI = Il;
    const bool diag = IJ.x == IJ.y;
    const float2 *__restrict__ T = (const float2 *)(ssm + (size_t)s * kC32HalfStageBytes);
    const float2 *__restrict__ fr = (const float2 *)(ssm + (size_t)s * kC32HalfStageBytes + kC32HalfBytes);
    const float2 *__restrict__ fc = fr + HR;
    float2 fcol[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) fcol[j] = fc[tj + 16 * j];
    if (h == 0)
#pragma unroll
      for (int j = 0; j < 4; ++j) cv[j] = 0.f;
    float rv[R];
#pragma unroll
    for (int i = 0; i < R; ++i) rv[i] = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int row = ti * R + i;
      const float2 fs = fr[row];
      float2 e[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) e[j] = T[row * kTile + tj + 16 * j];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float a = e[j].x, b = e[j].y;
        if (MODE == MODE_COLL) {
          const float t = c32_term(a, b, fs, fcol[j]);
          rv[i] = __fadd_rn(rv[i], t);
          if (!diag) cv[j] = __fsub_rn(cv[j], t);
        } else {  // 1/tau summands: row s: P_out + f_p d; column p (reverse channel): P_in - f_s d
          const float d = __fsub_rn(a, b);
          rv[i] = __fadd_rn(rv[i], __fmaf_rn(fcol[j].y, d, __fmaf_rn(fcol[j].x, d, b)));
          if (!diag) cv[j] = __fadd_rn(cv[j], __fmaf_rn(-fs.y, d, __fmaf_rn(-fs.x, d, a)));
        }
      }
    }
    // rows: the 16 lanes of a half-warp share them; lanes 8i .. 8i + 7 end with the total of row i
    f32_reduce_scatter<R, 8>(rv, lane);
    if ((tj & 7) == 0) tp[(long long)(IJ.x * kTile + h * HR + ti * R + (tj >> 3)) * nb + Jl] = rv[0];
    if (!diag && h == 1) {
      // columns of the whole tile: lanes tj and tj + 16 share them (one level), then the warps
      // (after the next unit's barrier)
      const bool up = lane & 16;
#pragma unroll
      for (int jk = 0; jk < 2; ++jk) {
        const int jo = jk + 2;
        const float kept = up ? cv[jo] : cv[jk], sent = up ? cv[jk] : cv[jo];
        colred[wid * kTile + tj + 16 * ((up ? 2 : 0) + jk)] = __fadd_rn(kept, __shfl_xor_sync(0xFFFFFFFFu, sent, 16));
      }
    }
  }
  if (!ok) {
    *err = 2;
    if (tid == 0) {
      for (int k = 0; k < NST; ++k) {
        const int uses = issued / NST + (k < issued % NST ? 1 : 0);
        if (uses > 0) mbar_wait(bars + k, (unsigned)((uses - 1) & 1));
      }
    }
  }
}

// The same FP32 pair coefficients as a row stream, for the batched rt-BTE (precision 2): entry
// e of the branch-merged rows holds C[e] = rounded (P_in, P_out) of (row state, partner colp[e]);
// one warp per item (a piece of one row), each lane two 4-entry groups per trip, partners'
// float-float f gathered through L1; part[item].x = sum of t(s, p) over the item.
template <typename IDX>
__global__ void __launch_bounds__(kBlock) k_stream_c32_rows(const Item *__restrict__ items, int nitems,
                                                            const float4 *__restrict__ C4,
                                                            const IDX *__restrict__ colp,
                                                            const float2 *__restrict__ fg,
                                                            Part4 *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < nitems; it += nwarps) {
    const Item I = items[it];
    const long long g0 = I.start >> 2;
    const int ng = I.len >> 2;
    const float2 fs = fg[I.row];
    float acc = 0.f, acc2 = 0.f;
    int g = lane;
    for (; g + 32 < ng; g += 64) {
      const long long q0 = g0 + g, q1 = q0 + 32;
      const uint4 c0 = partners4(colp, q0), c1 = partners4(colp, q1);
      const float4 x0 = __ldcs(C4 + 2 * q0), y0 = __ldcs(C4 + 2 * q0 + 1);
      const float4 x1 = __ldcs(C4 + 2 * q1), y1 = __ldcs(C4 + 2 * q1 + 1);
      acc = __fadd_rn(acc, c32_term(x0.x, x0.y, fs, fg[c0.x]));
      acc2 = __fadd_rn(acc2, c32_term(x1.x, x1.y, fs, fg[c1.x]));
      acc = __fadd_rn(acc, c32_term(x0.z, x0.w, fs, fg[c0.y]));
      acc2 = __fadd_rn(acc2, c32_term(x1.z, x1.w, fs, fg[c1.y]));
      acc = __fadd_rn(acc, c32_term(y0.x, y0.y, fs, fg[c0.z]));
      acc2 = __fadd_rn(acc2, c32_term(y1.x, y1.y, fs, fg[c1.z]));
      acc = __fadd_rn(acc, c32_term(y0.z, y0.w, fs, fg[c0.w]));
      acc2 = __fadd_rn(acc2, c32_term(y1.z, y1.w, fs, fg[c1.w]));
    }
    if (g < ng) {
      const long long q0 = g0 + g;
      const uint4 c0 = partners4(colp, q0);
      const float4 x0 = __ldcs(C4 + 2 * q0), y0 = __ldcs(C4 + 2 * q0 + 1);
      acc = __fadd_rn(acc, c32_term(x0.x, x0.y, fs, fg[c0.x]));
      acc = __fadd_rn(acc, c32_term(x0.z, x0.w, fs, fg[c0.y]));
      acc = __fadd_rn(acc, c32_term(y0.x, y0.y, fs, fg[c0.z]));
      acc = __fadd_rn(acc, c32_term(y0.z, y0.w, fs, fg[c0.w]));
    }
    acc = __fadd_rn(acc, acc2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, o));
    if (lane == 0) part[it] = make_part4((double)acc, 0.0, 0.0, 0.0);
  }
}

// C[e] = rounded (P_in, P_out) of n branch-merged float-float entries (A = P_in, B = D)
__global__ void k_pairs_c32(const float2 *__restrict__ A, const float2 *__restrict__ B, long long n,
                            float2 *__restrict__ C) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double pin = ff_to_double(A[e].x, A[e].y);
    C[e] = c32_round_pair(pin, pin + ff_to_double(B[e].x, B[e].y));
  }
}

// Epilogue of the C32 sweep: a 256-thread CTA takes SPC states; each warp adds the block
// partials of SPC / 8 states (lanes over the blocks in float-float, then one 32-lane float-float
// reduce-scatter of the SPC / 8 values), and warp 0 applies the prefactor and the RK4 stage
// arithmetic in FP64, one lane per state.
// pmap, binfo (batched tiles, else null): each state's padded row and the block table, whose
// .w gives the partner blocks of a state's system; nsp is then the number of states
template <int STAGE, bool RATE = false, int SPC = 32>
__global__ void __launch_bounds__(256) k_fin_c32(const float *__restrict__ tp, int nb, int nsp, int ns, double c,
                                                 const double *__restrict__ ysrc, double *__restrict__ out,
                                                 double *__restrict__ f, double *__restrict__ acc,
                                                 double *__restrict__ y, float2 *__restrict__ yff, double dt,
                                                 const int *__restrict__ pmap = nullptr,
                                                 const int4 *__restrict__ binfo = nullptr) {
  constexpr int SPW = SPC / 8, LPV = 32 / SPW;  // states per warp, lanes per state after the reduce-scatter
  __shared__ float2 tot[SPC];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int base = blockIdx.x * SPC;
  const int r0 = base + lane;
  FinIn in{0.0, 0.0, 0.0, 0.0};
  if (!RATE && wid == 0 && lane < SPC && r0 < ns) {
    if (STAGE >= 0) in.f = f[r0];
    if (STAGE >= 1) in.acc = acc[r0];
  }
  float2 v[SPW];
#pragma unroll
  for (int q = 0; q < SPW; ++q) {
    const int r = base + SPW * wid + q;
    v[q] = make_float2(0.f, 0.f);
    if (r < nsp) {
      const int pr = pmap ? pmap[r] : r, nbr = binfo ? binfo[pr / kTile].w : nb;
      const float *__restrict__ row = tp + (long long)pr * nb;
      for (int k = lane; k < nbr; k += 32) v[q] = ff_add(v[q], make_float2(row[k], 0.f));
    }
  }
  ff_reduce_scatter<SPW, 16>(v, lane);
  if ((lane & (LPV - 1)) == 0) tot[SPW * wid + lane / LPV] = v[0];
  __syncthreads();
  if (wid != 0 || lane >= SPC || r0 >= ns) return;
  const float2 Tt = tot[lane];
  const double I = c * ff_to_double(Tt.x, Tt.y);
  if (RATE) {
    out[r0] = I;
    return;
  }
  fin_stage<STAGE, false>(r0, I, in, out, f, acc, y, yff, dt, pmap ? pmap[r0] : r0);
}

}  // namespace dev
}  // namespace pb
