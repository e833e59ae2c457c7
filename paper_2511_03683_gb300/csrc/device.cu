// Device runtime of libpb.so: arena layout, upload, coefficient setup and the host
// drivers of the public compute calls (include/pb.h).  Kernels are in kernels.cuh.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "pb_internal.h"
#include "tiles32.cuh"

static_assert(pb::kRowPad == pb::dev::kEntryPad, "host row padding and the kernels' entry padding must agree");

using namespace pb;
using pb::dev::Item;
using pb::dev::Part4;

namespace {

constexpr size_t kAlign = 256;
constexpr int kFinBlock = 256;
// launch shapes of the FP32 tile sweep (pb_dev_opts.tile_sweep 2..6): stages per CTA and
// resident CTAs per SM
// (7, 8: half-tiles)
template <typename F>
void with_c32_shape(int shape, F &&fn) {
  using std::integral_constant;
  using std::false_type;
  using std::true_type;
  switch (shape) {
    case 3: fn(integral_constant<int, 3>(), integral_constant<int, 2>(), false_type()); break;
    case 4: fn(integral_constant<int, 2>(), integral_constant<int, 2>(), false_type()); break;
    case 5: fn(integral_constant<int, 4>(), integral_constant<int, 1>(), false_type()); break;
    case 6: fn(integral_constant<int, 6>(), integral_constant<int, 1>(), false_type()); break;
    case 7: fn(integral_constant<int, 3>(), integral_constant<int, 4>(), true_type()); break;
    case 8: fn(integral_constant<int, 4>(), integral_constant<int, 3>(), true_type()); break;
    default: fn(integral_constant<int, 2>(), integral_constant<int, 3>(), false_type()); break;
  }
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t rp, item_ptr, items, col, coefA, coefB, g2, wt, eps, kc, R, omega, tab, part, acc, y, yff, fstage, Fa, Fb,
      Fff, tau, invtau, red, scal, obs, g2lo, gstate, tab32, col16, rp_real, vjpG, g2tab, vecs, hcol, hg2, hA, hB, sc,
      entries, hitems, titems, t_item_ptr, err, citems, citem_ptr, cpart, ccoefA, ccoefB, sidx16, sidx32, pcstart,
      pcnt, srp, gitems, tiles, tcoef, tpart, g2d, gditems, gdptr, gacc, gaccg, trptr, trpart, total;
};

struct Plan {
  int64_t ns = 0, nchp = 0, nitems = 0;
  std::vector<int64_t> rp;       // padded row offsets [ns+1]
  std::vector<int32_t> item_ptr; // [ns+1]
  std::vector<Item> items;
  int item_ch = 0;
};

int default_item_channels(int64_t nchp, int sm_count, int ctas) {
  // (entries: channels, or state pairs of the branch-merged sweep)
  // enough items for ~4 per resident warp, 256..4096 channels each, multiple of 64
  const int64_t warps = (int64_t)sm_count * ctas * (dev::kBlock / 32);
  int64_t ic = nchp / std::max<int64_t>(1, warps * 4);
  ic = std::max<int64_t>(256, std::min<int64_t>(4096, ic));
  return (int)(ic / 64 * 64);
}

void plan_items(const std::vector<int64_t> &rp, int item_ch, std::vector<Item> &items, std::vector<int32_t> &ptr);

// Branch-merged sweep (FF and F64): one entry per state pair (s, p) = per run of equal partner
// in the CSR row, rows padded to kRowPad entries.  rp: padded entry offsets [ns+1].  Returns
// whether every row is complete (its partners are all nstate window states, in order).
bool pair_rows(const pb_channels *ch, std::vector<int64_t> &rp) {
  const int64_t ns = ch->nstate;
  rp.assign(ns + 1, 0);
  int complete = 1;
  // rows counted in parallel (each into rp[r + 1]), then the offsets summed in order
#pragma omp parallel for schedule(dynamic, 16) reduction(&& : complete)
  for (int64_t r = 0; r < ns; ++r) {
    int64_t runs = 0;
    for (int64_t c = ch->row_ptr[r]; c < ch->row_ptr[r + 1]; ++c)
      if (c == ch->row_ptr[r] || ch->col[c] != ch->col[c - 1]) ++runs;
    complete = complete && runs == ns;
    rp[r + 1] = (runs + kRowPad - 1) / kRowPad * kRowPad;
  }
  for (int64_t r = 0; r < ns; ++r) rp[r + 1] += rp[r];
  return complete != 0;
}

void plan_from_rp(const std::vector<int64_t> &rp, int item_ch, Plan &P) {
  P.ns = (int64_t)rp.size() - 1;
  P.item_ch = item_ch;
  P.rp = rp;
  plan_items(P.rp, item_ch, P.items, P.item_ptr);
  P.nchp = P.rp[P.ns];
  P.nitems = (int64_t)P.items.size();
}

void make_plan(const pb_channels *ch, int item_ch, Plan &P) {
  const int64_t ns = ch->nstate;
  P.ns = ns;
  P.item_ch = item_ch;
  P.rp.assign(ns + 1, 0);
  P.item_ptr.assign(ns + 1, 0);
  P.items.clear();
  for (int64_t r = 0; r < ns; ++r) {
    const int64_t len = ch->row_ptr[r + 1] - ch->row_ptr[r];
    const int64_t lenp = (len + kRowPad - 1) / kRowPad * kRowPad;
    P.rp[r + 1] = P.rp[r] + lenp;
    P.item_ptr[r] = (int32_t)P.items.size();
    if (lenp == 0) continue;
    const int64_t nchunks = lenp / kRowPad;  // 8-channel chunks
    const int64_t np = std::max<int64_t>(1, (lenp + item_ch - 1) / item_ch);
    int64_t off = 0;
    for (int64_t k = 0; k < np; ++k) {
      const int64_t chunks = nchunks / np + (k < nchunks % np ? 1 : 0);
      Item it;
      it.start = P.rp[r] + off;
      it.len = (int)(chunks * kRowPad);
      it.row = (int)r;
      if (it.len > 0) P.items.push_back(it);
      off += chunks * kRowPad;
    }
  }
  P.item_ptr[ns] = (int32_t)P.items.size();
  P.nchp = P.rp[ns];
  P.nitems = (int64_t)P.items.size();
}

// Paper layout (PB_VARIANT_PAPER): half list = the channels of row s with partner >= s;
// target list of state x = its half channels (+) and the half channels (s -> x), s < x (-),
// which by closure are as many as the full row of x.
struct PaperSizes {
  int64_t nh = 0, nhp = 0, nent = 0, nentp = 0;
};

PaperSizes paper_sizes(const pb_channels *ch) {
  PaperSizes z;
  for (int64_t r = 0; r < ch->nstate; ++r) {
    const int32_t *b = ch->col.data() + ch->row_ptr[r], *e = ch->col.data() + ch->row_ptr[r + 1];
    const int64_t h = e - std::lower_bound(b, e, (int32_t)r);
    z.nh += h;
    z.nhp += (h + kRowPad - 1) / kRowPad * kRowPad;
    z.nent += e - b;
    z.nentp += (e - b + kRowPad - 1) / kRowPad * kRowPad;
  }
  return z;
}

size_t coef_bytes(int variant) {
  switch (variant) {
    case PB_VARIANT_FF: return sizeof(float2);
    case PB_VARIANT_F64: return sizeof(double);
    default: return 0;
  }
}

// P: the channel plan; S: the sweep plan of the branch-merged variants (null: the sweep runs
// over channels and the channel-only regions are empty).
void plan_items(const std::vector<int64_t> &rp, int item_ch, std::vector<Item> &items, std::vector<int32_t> &ptr);

// Dense pair-major form of the mixed-precision sweep (pb_dev_opts.channel_per_lane 5, or 0 when
// the channel list fills at least 85% of the (row, branch, partner) slots): |g|^2 in one slot
// per (row, branch, partner), rows of npp partner slots (nstate rounded up to 32), items of
// `item` partners, about two per resident warp.
struct GDense {
  bool on = false;
  int npp = 0, nm = 0, item = 0;
  int64_t nitems = 0;
  size_t bytes = 0;
};
GDense gdense_for(const pb_channels *ch, const pb_dev_opts &o, int sm) {
  GDense g;
  const bool mixed = o.variant == PB_VARIANT_G32 || o.variant == PB_VARIANT_G16 || o.variant == PB_VARIANT_H16;
  if (!mixed || (o.channel_per_lane != 0 && o.channel_per_lane != 5)) return g;
  const int64_t ns = ch->nstate, nm = ch->nmodes;
  if (ns == 0 || nm == 0) return g;
  const int64_t npp = (ns + 31) / 32 * 32;
  const double slots = (double)ns * (double)nm * (double)npp;
  if (o.channel_per_lane == 0 && (double)ch->row_ptr[ns] < 0.85 * slots) return g;
  g.on = true;
  g.npp = (int)npp;
  g.nm = (int)nm;
  const int64_t warps = (int64_t)sm * 32;
  const int64_t item = (ns * npp / (2 * warps) + 31) / 32 * 32;
  g.item = (int)std::max<int64_t>(256, std::min<int64_t>(item, npp));
  g.nitems = ns * std::max<int64_t>(1, (npp + g.item - 1) / g.item);
  g.bytes = (size_t)(o.variant == PB_VARIANT_G32 ? 4 : 2) * (size_t)slots;
  return g;
}

// work items of the branch-merged |g|^2 gradient: the sweep rows in pieces of at most one warp
// width of entries (plan_items never exceeds item_ch)
int64_t grad_chunks(const std::vector<int64_t> &rp) {
  std::vector<Item> it;
  std::vector<int32_t> ptr;
  plan_items(rp, dev::kWarpChunk, it, ptr);
  return (int64_t)it.size();
}

// symmetric tiles of the complete-row FF sweep: nb blocks of kTile states, nt = nb(nb+1)/2 tiles
struct TileDims {
  int nb = 0, nt = 0, nsp = 0;
};
TileDims tile_dims(int64_t ns) {
  TileDims t;
  t.nb = (int)((ns + dev::kTile - 1) / dev::kTile);
  t.nt = t.nb * (t.nb + 1) / 2;
  t.nsp = t.nb * dev::kTile;
  return t;
}

// tile_entry: bytes per pair of the symmetric tiles (16 float-float, 8 for the FP32 tiles of C32)
Layout make_layout(const pb_channels *ch, const Plan &P, const Plan *S, int variant, bool transport,
                   int nfin_blocks, bool sym = false, const GDense &gd = GDense(), bool gacc = false,
                   size_t tile_entry = sizeof(float4), int tr_nseg = 0) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + std::max<size_t>(bytes, 1));
    return at;
  };
  const size_t ns = (size_t)P.ns, nchp = (size_t)P.nchp;
  const Plan &W = S ? *S : P;  // the sweep plan
  const size_t nsw = (size_t)W.nchp;
  L.rp = take(sizeof(int64_t) * (ns + 1));
  L.item_ptr = take(sizeof(int32_t) * (ns + 1));
  L.items = take(sizeof(Item) * W.nitems);
  L.citem_ptr = take(S ? sizeof(int32_t) * (ns + 1) : 0);
  L.citems = take(S ? sizeof(Item) * P.nitems : 0);
  L.cpart = take(S ? sizeof(Part4) * P.nitems : 0);
  L.col = take(sizeof(uint32_t) * nchp);
  L.g2 = take(sizeof(double) * nchp);
  L.coefA = take(coef_bytes(variant) * nsw);
  L.coefB = take(coef_bytes(variant) * nsw);
  L.ccoefA = take(S ? coef_bytes(variant) * nchp : 0);
  L.ccoefB = take(S ? coef_bytes(variant) * nchp : 0);
  L.sidx16 = take(S && ns <= 65536 ? sizeof(uint16_t) * nsw : 0);
  L.sidx32 = take(S && ns > 65536 ? sizeof(uint32_t) * nsw : 0);
  L.pcstart = take(S ? sizeof(int64_t) * nsw : 0);
  L.pcnt = take(S ? nsw : 0);
  L.srp = take(S ? sizeof(int64_t) * (ns + 1) : 0);
  L.gitems = take(S ? sizeof(Item) * (size_t)grad_chunks(S->rp) : 0);
  L.gacc = take(S && gacc && variant == PB_VARIANT_FF ? sizeof(float4) * nsw : 0);
  L.gaccg = take(gacc && (variant == PB_VARIANT_G32 || variant == PB_VARIANT_G16 || variant == PB_VARIANT_H16) ? 3 * sizeof(double) * (size_t)ns * (size_t)ns : 0);
  const TileDims td = tile_dims((int64_t)ns);
  L.tiles = take(sym ? sizeof(int2) * td.nt : 0);
  L.tcoef = take(sym ? tile_entry * (size_t)td.nt * dev::kTile * dev::kTile : 0);
  L.tpart = take(sym ? sizeof(float4) * (size_t)td.nb * td.nsp : 0);
  L.wt = take(transport ? sizeof(float2) * nsw : 0);
  L.eps = take(sizeof(double) * ns);
  L.kc = take(sizeof(short4) * ns);
  L.R = take(sizeof(double) * ns);
  L.omega = take(sizeof(double) * (size_t)ch->nq * ch->nmodes);
  L.tab = take(sizeof(double2) * (size_t)ch->nq * ch->nmodes);
  L.acc = take(sizeof(double) * ns);
  L.y = take(sizeof(double) * ns);
  L.yff = take(sizeof(float2) * ns);
  L.fstage = take(sizeof(double) * ns);
  L.Fa = take(transport ? sizeof(double) * 3 * ns : 0);
  L.Fb = take(transport ? sizeof(double) * 3 * ns : 0);
  L.Fff = take(transport ? sizeof(float2) * 3 * ns : 0);
  L.tau = take(sizeof(double) * ns);
  L.invtau = take(sizeof(double) * ns);
  L.red = take(sizeof(double2) * (size_t)nfin_blocks);
  L.scal = take(sizeof(double) * 8);
  L.obs = take(sizeof(double) * 8);
  L.err = take(sizeof(int) * 4);
  const bool mixed = variant == PB_VARIANT_G32 || variant == PB_VARIANT_G16 || variant == PB_VARIANT_H16;
  L.g2lo = take(mixed ? (variant == PB_VARIANT_G32 ? 4 : 2) * nchp : 0);
  L.gstate = take(mixed ? 16 * ns : 0);
  auto rad = [](int n) { return (size_t)(n > 1 ? 2 * n : 1); };
  L.tab32 = take(mixed ? sizeof(float2) * rad(ch->nk[0]) * rad(ch->nk[1]) * rad(ch->nk[2]) * ch->nmodes : 0);
  L.col16 = take(ns <= 65536 ? sizeof(uint16_t) * nchp : 0);
  PaperSizes z;
  if (variant == PB_VARIANT_PAPER) z = paper_sizes(ch);
  const int64_t nhi = (variant == PB_VARIANT_PAPER) ? z.nhp / kRowPad + (int64_t)ns : 0;  // upper bound of items
  L.hcol = take(sizeof(uint32_t) * z.nhp);
  L.hg2 = take(sizeof(double) * z.nhp);
  L.hA = take(sizeof(float2) * z.nhp);
  L.hB = take(sizeof(float2) * z.nhp);
  L.sc = take(sizeof(float2) * (z.nhp + 8));
  L.entries = take(sizeof(int32_t) * z.nentp);
  L.hitems = take(sizeof(Item) * nhi);
  L.titems = take(sizeof(Item) * ((variant == PB_VARIANT_PAPER) ? z.nentp / kRowPad + (int64_t)ns : 0));
  L.t_item_ptr = take(sizeof(int32_t) * (ns + 1));
  L.part = take(sizeof(Part4) * std::max<int64_t>(std::max<int64_t>(W.nitems, gd.nitems),
                                                  (variant == PB_VARIANT_PAPER) ? z.nentp / kRowPad + (int64_t)ns : 0));
  L.g2d = take(gd.on ? gd.bytes : 0);
  L.gditems = take(gd.on ? sizeof(Item) * (size_t)gd.nitems : 0);
  L.gdptr = take(gd.on ? sizeof(int32_t) * (ns + 1) : 0);
  L.rp_real = take(sizeof(int64_t) * (ns + 1));
  L.vjpG = take(sizeof(float2) * 3 * ns);
  L.g2tab = take(sizeof(float4) * 2 * 4 * ns);
  L.vecs = take(sizeof(double) * 9 * ns);
  L.trptr = take(tr_nseg ? sizeof(int32_t) * (ns + 1) : 0);
  L.trpart = take(tr_nseg ? sizeof(Part4) * ns * (size_t)tr_nseg : 0);
  L.total = o;
  return L;
}

// Segments of the row-block transport sweep (k_stream_tr_rows, pb_dev_opts.transport_gather 7)
// over complete rows: enough
// (row block, segment) items to give every warp of one wave about one item, each segment at most
// dev::kTrSegMax partners (the lazy float-float sums' bound) and, where the rows allow, at least
// 256; seglen a multiple of 32.  nseg = 0 where the sweep is not asked for or does not apply (rows not
// complete and branch-merged, another variant, or F of every state and the weight rings too large
// for shared memory).
struct TrRows {
  int nseg = 0, seglen = 0;
};
TrRows tr_rows_for(int64_t ns, int sm, bool transport, bool merged, bool complete, int variant,
                   const pb_dev_opts &o) {
  TrRows t;
  if (!transport || o.transport_gather != 7 || !merged || !complete || variant != PB_VARIANT_FF ||
      o.dense_rows == 2 || ns < 1 ||
      ns > (int64_t)1 << 20 || dev::tr_rows_smem((int)ns) > (size_t)227 * 1024)
    return t;
  const int64_t nwarps = (int64_t)std::max(sm, 1) * (dev::kTrThreads / 32);
  const int64_t nblk = (ns + dev::kTrRows - 1) / dev::kTrRows;
  int64_t nseg = std::max<int64_t>((ns + dev::kTrSegMax - 1) / dev::kTrSegMax,
                                   std::min<int64_t>(nwarps / nblk, (ns + 255) / 256));
  nseg = std::max<int64_t>(nseg, 1);
  const int64_t seglen = ((ns + nseg - 1) / nseg + 31) / 32 * 32;
  t.seglen = (int)seglen;
  t.nseg = (int)((ns + seglen - 1) / seglen);
  return t;
}

int cuda_fail(cudaError_t e, const char *what) {
  return set_error(PB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PB_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);         \
  } while (0)

#define PB_LAUNCHED(what)                                       \
  do {                                                          \
    cudaError_t e_ = cudaGetLastError();                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);          \
  } while (0)

}  // namespace

namespace {
// fn(T *) with T the |g|^2 storage type of a mixed-precision variant (G32, G16, H16; the
// callers check pb_dev::mixed() first, and other variants call nothing)
template <typename F>
void with_g2t(int variant, F &&fn) {
  if (variant == PB_VARIANT_G32) fn((float *)nullptr);
  else if (variant == PB_VARIANT_G16) fn((__nv_bfloat16 *)nullptr);
  else if (variant == PB_VARIANT_H16) fn((__half *)nullptr);
}

// Mixed-precision lane-sweep shapes (pb_dev_opts.channel_per_lane): 1 = 512 threads, three
// CTAs per SM; 3 = the same with an L2 prefetch two trips ahead; 4 = one 1024-thread CTA per
// SM with the next trip's stream words in registers.
template <typename G2T>
void set_lane_smem(int bytes) {
  using namespace pb::dev;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaFuncSetAttribute(k_stream_g_lane<MODE_COLL, G2T, 0, 512, false>, A, bytes);
  cudaFuncSetAttribute(k_stream_g_lane<MODE_RATE, G2T, 0, 512, false>, A, bytes);
  cudaFuncSetAttribute(k_stream_g_lane<MODE_COLL, G2T, 2, 512, false>, A, bytes);
  cudaFuncSetAttribute(k_stream_g_lane<MODE_RATE, G2T, 2, 512, false>, A, bytes);
  cudaFuncSetAttribute(k_stream_g_lane<MODE_COLL, G2T, 0, 1024, true>, A, bytes);
  cudaFuncSetAttribute(k_stream_g_lane<MODE_RATE, G2T, 0, 1024, true>, A, bytes);
}

template <int PF, int NT, bool RP, typename G2T>
void launch_g_lane_t(bool coll, int grid, size_t smem, cudaStream_t st, const pb::dev::Item *items, int n,
                     const pb::dev::GGeom &g, const G2T *g2, const uint4 *gstate, int ns, pb::dev::Part4 *part) {
  using namespace pb::dev;
  if (coll) k_stream_g_lane<MODE_COLL, G2T, PF, NT, RP><<<grid, NT, smem, st>>>(items, n, g, g2, gstate, ns, part);
  else      k_stream_g_lane<MODE_RATE, G2T, PF, NT, RP><<<grid, NT, smem, st>>>(items, n, g, g2, gstate, ns, part);
}

// grid512: the grid of 512-thread CTAs; the 1024-thread shape runs one CTA per SM
template <typename G2T>
void launch_g_lane(int shape, bool coll, int grid512, int sm_count, size_t smem, cudaStream_t st,
                   const pb::dev::Item *items, int n, const pb::dev::GGeom &g, const G2T *g2, const uint4 *gstate,
                   int ns, pb::dev::Part4 *part) {
  if (shape == 4)
    launch_g_lane_t<0, 1024, true>(coll, std::max(1, std::min(sm_count, (n * 32 + 1023) / 1024)), smem, st, items, n,
                                   g, g2, gstate, ns, part);
  else if (shape == 3)
    launch_g_lane_t<2, 512, false>(coll, grid512, smem, st, items, n, g, g2, gstate, ns, part);
  else
    launch_g_lane_t<0, 512, false>(coll, grid512, smem, st, items, n, g, g2, gstate, ns, part);
}
}  // namespace

struct pb_dev {
  int variant = 0;
  int64_t ns = 0, nch = 0, nchp = 0, nitems = 0;
  int nk[3] = {0, 0, 0};
  int nmodes = 0;
  int64_t nq = 0;
  double T = 0, sigma = 0, c = 0;
  int sm_count = 0, ctas = 4, item_ch = 0;
  bool transport = false;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  Layout L{};
  // device views
  int64_t *rp = nullptr;
  int32_t *item_ptr = nullptr;
  Item *items = nullptr;
  uint32_t *col = nullptr;
  double *g2 = nullptr;
  void *coefA = nullptr, *coefB = nullptr;
  float2 *wt = nullptr;
  double *eps = nullptr;
  short4 *kc = nullptr;
  double *R = nullptr;
  double *omega = nullptr;
  double2 *tab = nullptr;
  Part4 *part = nullptr;
  double *acc = nullptr, *y = nullptr, *fstage = nullptr;
  float2 *yff = nullptr;
  double *Fa = nullptr, *Fb = nullptr;
  float2 *Fff = nullptr;
  double *tau = nullptr, *invtau = nullptr;
  double2 *red = nullptr;
  double *scal = nullptr, *obs = nullptr;
  int *err = nullptr;       // device error word (bounded waits that gave up)
  bool bulk = false;        // collision sweep through TMA bulk copies
  int bulk_cap = 0;         // largest work item (channels), the bulk stage capacity
  size_t bulk_smem = 0;
  void *g2lo = nullptr;     // |g|^2 in FP32 or BF16 (mixed-precision variants)
  // dense pair-major mixed-precision sweep (GDense)
  bool gdense = false;
  int gd_npp = 0, gd_nitems = 0;
  size_t gd_bytes = 0;
  void *g2d = nullptr;
  Item *gd_items = nullptr;
  int32_t *gd_item_ptr = nullptr;
  uint4 *gstate = nullptr;  // per-state records of the mixed-precision sweep (eps, f, grid index)
  bool vjp_g_ok = false;    // the mixed-precision adjoint's 20 bytes per state fit in shared memory
  float2 *tab32 = nullptr;  // padded-grid (hbar w, N) in FP32
  uint16_t *col16 = nullptr;  // 16-bit partner indices (nstate <= 65536), else null
  // branch-merged sweep (FF, F64): items/item_ptr/part/coefA/coefB/wt above are per state
  // pair; the per-channel plan and coefficients below feed the setup and the |g|^2 gradient.
  // Without merging the c* views alias the sweep's and sidx* alias col16/col.
  bool merged = false;
  int64_t ncitems = 0, nsw = 0;   // channel-plan items; sweep entries (padded)
  Item *citems = nullptr;
  int32_t *citem_ptr = nullptr;
  Part4 *cpart = nullptr;
  void *ccoefA = nullptr, *ccoefB = nullptr;
  uint16_t *sidx16 = nullptr;     // sweep partner indices (16-bit when nstate <= 65536)
  uint32_t *sidx32 = nullptr;
  int64_t *pcstart = nullptr;     // first channel of each sweep entry
  uint8_t *pcnt = nullptr;        // channels of each sweep entry
  // complete rows (every row holds every window state, in order): the FF collision and the
  // transport sweeps take each entry's partner from its position and stream no index
  bool dense = false;
  int64_t *srp = nullptr;         // first sweep entry of every row [ns+1]
  Item *gitems = nullptr;         // the sweep rows in pieces of <= 32 entries (|g|^2 gradient)
  float4 *gacc = nullptr;         // deferred |g|^2 gradient: (u, v) float-float per sweep entry
  double *gaccg = nullptr;        // deferred mixed |g|^2 gradient: W, U, V per (state, partner), FP64
  size_t gaccg_bytes() const { return 3 * sizeof(double) * (size_t)ns * (size_t)ns; }
  int ngitems = 0;
  // symmetric tiles (complete rows, FF): the collision and rate sweeps stream the upper block
  // triangle of the pair matrix once and add each tile to its rows and to its columns
  bool sym = false;
  int sym_nt = 0;  // threads of the bulk-copy tile sweep's CTA (0: the global-load tile sweep)
  TileDims td;
  int2 *tiles = nullptr;
  float4 *tcoef = nullptr;
  float4 *tpart = nullptr;
  // PB_VARIANT_C32: the FF device whose tiles hold FP32 (P_in, P_out) (tiles32.cuh); its
  // partials in tpart are (N, Bd, L, Ld) per (state, block)
  bool sym_half = false;  // the float-float tile sweep in half-tiles (tile_sweep 3)
  int half_cps = 3;       // its resident CTAs per SM: 3 (two stages each) or 2 (three stages)
  bool c32 = false;
  int c32_shape = 2;  // pb_dev_opts.tile_sweep: the launch shape (with_c32_shape)
  bool complete = false;  // every row holds every state (tiles filled by position, else scattered)
  // the next tile sweep takes the tile list from its end (the RK4 stages alternate, so that each
  // sweep starts on the tiles the previous one left in L2)
  int rev = 0;
  // pb_iter_transport: page-locked host copies of the residual numbers of two successive
  // passes (allocated on the first solve), so that the next pass runs while one is checked
  double *hres = nullptr;
  cudaEvent_t hres_ev[2] = {nullptr, nullptr};
  float2 *tc32 = nullptr;
  int64_t *rp_real = nullptr;  // unpadded CSR row offsets [ns+1]
  float2 *vjpG = nullptr;      // adjoint gather table [ns][3]
  int tr_nseg = 0, tr_seglen = 0;  // row-block transport sweep: segments per row, partners per segment
  int32_t *trptr = nullptr;        // its partial ranges per row (r * tr_nseg) for the finaliser
  Part4 *trpart = nullptr;         // its (row, segment) partials [ns][tr_nseg]
  size_t smem_Frows = 0;           // its shared-memory F
  float4 *g2tab = nullptr;     // |g|^2-gradient stage table [4 stages][ns][2]
  double *vecs = nullptr;      // 9 scratch vectors of nstate doubles (adjoint stages, the step's f)
  // paper layout (PB_VARIANT_PAPER)
  uint32_t *hcol = nullptr;
  double *hg2 = nullptr;
  float2 *hA = nullptr, *hB = nullptr, *sc = nullptr;
  int32_t *entries = nullptr, *t_item_ptr = nullptr;
  Item *hitems = nullptr, *titems = nullptr;
  int64_t nhitems = 0, ntitems = 0, nh = 0, nhp = 0, nent = 0;
  int rad[3] = {1, 1, 1};   // padded-grid radices of the FP32 phonon table
  int nfin_blocks = 0;
  size_t smem_f = 0;      // dynamic smem of the f staging (0 = gather from global)
  size_t smem_F = 0;      // dynamic smem of the transport F staging
  int ctas_tr = 1;        // resident transport CTAs per SM
  size_t smem_G = 0;      // dynamic smem of the adjoint gather table
  bool tr_lane = true;    // L1-gather transport with consecutive lanes on consecutive channels
  int tr_shape = 3;       // its launch shape (pb_dev_opts.transport_gather 3..6)
  size_t smem_F1k = 0;    // shared-memory F of the 1024-thread transport shape
  bool g_lane = true;     // mixed-precision sweep with consecutive lanes on consecutive channels
  int g_shape = 1;        // its launch shape (pb_dev_opts.channel_per_lane: 1, 3 or 4)
  // RK4 graph cache
  cudaStream_t cap = nullptr;
  cudaGraphExec_t rk_exec = nullptr;
  cudaGraphExec_t rk_exec_in = nullptr;  // the same step preceded by the stage-input conversion of f
  // graphs of the short launch sequences of pb_collision, pb_scatter_rates and
  // pb_transport_iterate, one per call kind and argument set, the last kGraphs kept
  static constexpr int kGraphs = 12;
  struct CallGraph {
    int kind = 0;
    const void *a = nullptr, *b = nullptr, *c = nullptr, *e = nullptr;
    cudaGraphExec_t exec = nullptr;
  } cg[kGraphs];
  int cg_next = 0;
  void drop_call_graphs() {
    for (auto &g : cg) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      g = CallGraph{};
    }
  }
  double *rk_f = nullptr;
  double rk_dt = 0.0;
  pb::dev::ChanGeom geom() const {
    pb::dev::ChanGeom g;
    g.col = col;
    g.g2 = g2;
    g.eps = eps;
    g.kc = kc;
    g.tab = tab;
    g.N1 = nk[0];
    g.N2 = nk[1];
    g.N3 = nk[2];
    g.nmodes = nmodes;
    g.inv2s2 = 1.0 / (2.0 * sigma * sigma);
    g.norm = 1.0 / (std::sqrt(2.0 * kPi) * sigma);
    return g;
  }
  bool mixed() const { return variant == PB_VARIANT_G32 || variant == PB_VARIANT_G16 || variant == PB_VARIANT_H16; }
  // mixed variants: the stored |g|^2 is s2 |g|^2 (a power of two; 1 but for FP16), so the
  // prefactor of their sums is c gnorm / s2
  double g2s = 1.0;
  double gscale() const { return c * gnorm() / g2s; }
  // the work items whose partials the forward sweeps write (collision, rates, RK4 stages)
  const int32_t *fwd_item_ptr() const { return gdense ? gd_item_ptr : item_ptr; }
  pb::dev::GGeom ggeom() const {
    pb::dev::GGeom g;
    g.col = col;
    g.tabp = tab32;
    const int n1 = rad[0] > 1 ? nk[0] : 0, n2 = rad[1] > 1 ? nk[1] : 0, n3 = rad[2] > 1 ? nk[2] : 0;
    g.cpad = ((n1 * rad[1] + n2) * rad[2] + n3) * nmodes;
    g.k2 = (float)(-1.4426950408889634 / (2.0 * sigma * sigma));
    return g;
  }
  double gnorm() const { return 1.0 / (std::sqrt(2.0 * kPi) * sigma); }
  int stream_grid(int per_sm) const {
    const int64_t need = (nitems * 32 + dev::kBlock - 1) / dev::kBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sm_count * per_sm));
  }
  int chan_grid(int per_sm) const {
    const int64_t need = (ncitems * 32 + dev::kBlock - 1) / dev::kBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sm_count * per_sm));
  }
};

namespace {

int check_device(int *sm_count) {
  int devid = 0, major = 0, minor = 0;
  cudaError_t e = cudaGetDevice(&devid);
  if (e != cudaSuccess) return set_error(PB_EDEVICE, "no CUDA device: %s", cudaGetErrorString(e));
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, devid);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, devid);
  if (major != 10 || minor != 3)
    return set_error(PB_EDEVICE, "libpb.so is built for sm_103a only; device is sm_%d%d", major, minor);
  PB_CUDA(cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, devid));
  return PB_OK;
}

int resolve_opts(const pb_channels *ch, const pb_dev_opts *opts, int sm_count, pb_dev_opts &o) {
  pb_dev_opts d{};
  if (opts) d = *opts;
  if (d.variant < PB_VARIANT_FF || d.variant > PB_VARIANT_C32)
    return set_error(PB_EINVAL, "pb_dev: variant %d is not available in this build", d.variant);
  if (d.merge_branches < 0 || d.merge_branches > 2) return set_error(PB_EINVAL, "pb_dev: merge_branches must be 0..2");
  if (d.dense_rows < 0 || d.dense_rows > 3) return set_error(PB_EINVAL, "pb_dev: dense_rows must be 0..3");
  if (d.tile_sweep < 0 || d.tile_sweep > 8 || (d.tile_sweep > 3 && d.variant != PB_VARIANT_C32))
    return set_error(PB_EINVAL, "pb_dev: tile_sweep must be 0..3 (0..8 for the FP32 coefficient tiles)");
  if (d.adjoint < 0 || d.adjoint > 1) return set_error(PB_EINVAL, "pb_dev: adjoint must be 0 or 1");
  // automatic: the half-tile ring (measured 38.8 us per 40^3 sweep against 42.6 us for whole tiles);
  // for C32 its own default shape
  if (d.tile_sweep == 0) d.tile_sweep = d.variant == PB_VARIANT_C32 ? 2 : 3;
  if (d.variant == PB_VARIANT_C32 && (d.tile_sweep == 1 || d.stream_mode == 2 || d.merge_branches == 2 ||
                                      d.dense_rows == 1 || d.dense_rows == 2))
    return set_error(PB_EINVAL, "pb_dev: the FP32 coefficient tiles (C32) need branch merging and the symmetric "
                                "bulk-copy tile sweep (merge_branches 0/1, dense_rows 0/3, tile_sweep 0/2..6, "
                                "stream_mode 0/1)");
  // measured best on GB300 at 40^3: 3 CTAs per SM for one entry per channel, 4 for the
  // branch-merged sweep (whose stream is six times shorter)
  const bool merged = (d.variant == PB_VARIANT_FF || d.variant == PB_VARIANT_F64 || d.variant == PB_VARIANT_C32) &&
                      d.merge_branches != 2;
  if (d.ctas_per_sm <= 0) d.ctas_per_sm = merged ? 4 : 3;
  if (d.ctas_per_sm > 8) return set_error(PB_EINVAL, "pb_dev: ctas_per_sm must be <= 8");
  if (d.stream_mode < 0 || d.stream_mode > 2) return set_error(PB_EINVAL, "pb_dev: stream_mode must be 0..2");
  if (d.channel_per_lane < 0 || d.channel_per_lane > 5)
    return set_error(PB_EINVAL, "pb_dev: channel_per_lane must be 0..5");
  if (d.transport_gather < 0 || d.transport_gather > 7 || d.transport_ctas < 0 || d.transport_ctas > 8)
    return set_error(PB_EINVAL, "pb_dev: transport_gather must be 0..7 and transport_ctas 0..8");
  if (d.item_channels < 0 || d.item_channels % 64 != 0)
    return set_error(PB_EINVAL, "pb_dev: item_channels must be a non-negative multiple of 64");
  if (d.item_channels == 0 && d.stream_mode == 2) d.item_channels = 2048;  // bulk ring fits shared memory
  if (d.item_channels == 0) {
    int64_t nchp = 0;
    for (int64_t r = 0; r < ch->nstate; ++r)
      nchp += (ch->row_ptr[r + 1] - ch->row_ptr[r] + kRowPad - 1) / kRowPad * kRowPad;
    d.item_channels = default_item_channels(nchp, sm_count, d.ctas_per_sm);
  }
  o = d;
  return PB_OK;
}

bool merge_for(const pb_dev_opts &o) {
  return (o.variant == PB_VARIANT_FF || o.variant == PB_VARIANT_F64) && o.merge_branches != 2;
}

// whether the symmetric tiles of ns states stream at most 0.7 of the bytes of a branch-merged
// row stream of nsw entries (float-float P_in and D and a 16- or 32-bit partner index): rows
// that miss some partners, but not many
bool tiles_pay(int64_t ns, int64_t nsw) {
  const double nb = (double)((ns + dev::kTile - 1) / dev::kTile);
  const double tile_bytes = nb * (nb + 1) / 2 * dev::kTile * dev::kTile * 16.0;
  const double row_bytes = (double)nsw * (16.0 + (ns <= 65536 ? 2.0 : 4.0));
  return tile_bytes <= 0.7 * row_bytes;
}

// symmetric tiles: FF, branch-merged, a list verified closed under reversal (the entry of (s, p)
// serves (p, s) with P_in and P_out swapped); dense_rows 3, or automatic (0) on complete rows or
// when the tiles stream fewer bytes than the rows (pays)
bool sym_for(const pb_dev_opts &o, bool merged, bool complete, bool closed, bool pays) {
  if (!(merged && closed && o.variant == PB_VARIANT_FF && o.stream_mode != 2)) return false;
  return o.dense_rows == 3 || (o.dense_rows == 0 && (complete || pays));
}

// work-item size of the branch-merged sweep: the caller's, the bulk ring's, or the default
int sweep_item_size(const pb_dev_opts *user, const pb_dev_opts &o, const std::vector<int64_t> &rp, int sm) {
  if (user && user->item_channels > 0) return user->item_channels;
  if (o.stream_mode == 2) return 2048;
  // about two items per resident warp, each row cut into equal pieces (256..4096 entries):
  // the per-item reduction and the finaliser's partial sums cost more than the tail of the
  // last wave at this stream length
  const int64_t ns = (int64_t)rp.size() - 1, nsw = rp.back();
  int64_t rows = 0;
  for (int64_t r = 0; r < ns; ++r) rows += rp[r + 1] > rp[r];
  if (rows == 0) return 256;
  const int64_t warps = (int64_t)sm * o.ctas_per_sm * (dev::kBlock / 32);
  const int64_t per_row = std::max<int64_t>(1, (2 * warps + rows / 2) / rows);  // pieces per row
  int64_t ic = (nsw / rows + per_row - 1) / per_row;
  ic = std::max<int64_t>(256, std::min<int64_t>(4096, (ic + 63) / 64 * 64));
  return (int)ic;
}

// channel plan P and, for the branch-merged variants, the sweep plan S (complete: every row
// holds every window state)
bool make_plans(const pb_channels *ch, const pb_dev_opts *user, const pb_dev_opts &o, int sm, Plan &P, Plan &S,
                bool *complete = nullptr) {
  make_plan(ch, o.item_channels, P);
  if (complete) *complete = false;
  if (!merge_for(o)) return false;
  std::vector<int64_t> rp;
  const bool c = pair_rows(ch, rp);
  if (complete) *complete = c;
  plan_from_rp(rp, sweep_item_size(user, o, rp, sm), S);
  return true;
}

}  // namespace

namespace {

void plan_items(const std::vector<int64_t> &rp, int item_ch, std::vector<Item> &items, std::vector<int32_t> &ptr) {
  const int64_t ns = (int64_t)rp.size() - 1;
  items.clear();
  ptr.assign(ns + 1, 0);
  for (int64_t r = 0; r < ns; ++r) {
    ptr[r] = (int32_t)items.size();
    const int64_t lenp = rp[r + 1] - rp[r];
    if (lenp == 0) continue;
    const int64_t chunks = lenp / kRowPad, np = std::max<int64_t>(1, (lenp + item_ch - 1) / item_ch);
    int64_t off = 0;
    for (int64_t k = 0; k < np; ++k) {
      const int64_t c = chunks / np + (k < chunks % np ? 1 : 0);
      if (c > 0) {
        Item it;
        it.start = rp[r] + off;
        it.len = (int)(c * kRowPad);
        it.row = (int)r;
        items.push_back(it);
      }
      off += c * kRowPad;
    }
  }
  ptr[ns] = (int32_t)items.size();
}

// Half list, per-channel coefficients of the half list, and the signed target layer.
int paper_setup(pb_dev *d, const pb_channels *ch, int item_ch, cudaStream_t st) {
  const int64_t ns = ch->nstate;
  std::vector<int64_t> hstart(ns), hlen(ns), hrp(ns + 1, 0), trp(ns + 1, 0);
  for (int64_t r = 0; r < ns; ++r) {
    const int32_t *b = ch->col.data() + ch->row_ptr[r], *e = ch->col.data() + ch->row_ptr[r + 1];
    const int32_t *lo = std::lower_bound(b, e, (int32_t)r);
    hstart[r] = lo - ch->col.data();
    hlen[r] = e - lo;
    hrp[r + 1] = hrp[r] + (hlen[r] + kRowPad - 1) / kRowPad * kRowPad;
    const int64_t full = e - b;
    trp[r + 1] = trp[r] + (full + kRowPad - 1) / kRowPad * kRowPad;
  }
  const int64_t nhp = hrp[ns], nentp = trp[ns];
  std::vector<uint32_t> hcol((size_t)nhp);
  std::vector<double> hg2((size_t)nhp, 0.0);
  std::vector<int32_t> ent((size_t)nentp, (int32_t)nhp);  // padding entries read the zero slot
  std::vector<int64_t> fill(ns, 0);
  int64_t nh = 0, nent = 0;
  for (int64_t r = 0; r < ns; ++r) {
    for (int64_t k = 0; k < hlen[r]; ++k) {
      const int64_t c = hstart[r] + k, h = hrp[r] + k;
      const int32_t p = ch->col[c];
      hcol[h] = (uint32_t)p | ((uint32_t)ch->nu[c] << kPartnerBits);
      hg2[h] = ch->g2[c];
      ent[trp[r] + fill[r]++] = (int32_t)h;
      ++nent;
      if (p != (int32_t)r) {
        ent[trp[p] + fill[p]++] = (int32_t)(h | (int64_t)0x80000000LL);
        ++nent;
      }
      ++nh;
    }
    for (int64_t k = hlen[r]; k < hrp[r + 1] - hrp[r]; ++k) hcol[hrp[r] + k] = (uint32_t)r;
  }
  std::vector<Item> hitems, titems;
  std::vector<int32_t> hptr, tptr;
  plan_items(hrp, item_ch, hitems, hptr);
  plan_items(trp, item_ch, titems, tptr);
  PB_CUDA(cudaMemcpyAsync(d->hcol, hcol.data(), sizeof(uint32_t) * nhp, cudaMemcpyHostToDevice, st));
  PB_CUDA(cudaMemcpyAsync(d->hg2, hg2.data(), sizeof(double) * nhp, cudaMemcpyHostToDevice, st));
  PB_CUDA(cudaMemcpyAsync(d->entries, ent.data(), sizeof(int32_t) * nentp, cudaMemcpyHostToDevice, st));
  PB_CUDA(cudaMemcpyAsync(d->hitems, hitems.data(), sizeof(Item) * hitems.size(), cudaMemcpyHostToDevice, st));
  PB_CUDA(cudaMemcpyAsync(d->titems, titems.data(), sizeof(Item) * titems.size(), cudaMemcpyHostToDevice, st));
  PB_CUDA(cudaMemcpyAsync(d->t_item_ptr, tptr.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice, st));
  PB_CUDA(cudaMemsetAsync(d->sc, 0, sizeof(float2) * (nhp + 8), st));
  d->nhitems = (int64_t)hitems.size();
  d->ntitems = (int64_t)titems.size();
  d->nh = nh;
  d->nhp = nhp;
  d->nent = nent;
  pb::dev::ChanGeom g = d->geom();
  g.col = d->hcol;
  g.g2 = d->hg2;
  const int64_t need = (d->nhitems * 32 + dev::kBlock - 1) / dev::kBlock;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)d->sm_count * 8));
  dev::k_coef<true><<<grid, dev::kBlock, 0, st>>>(d->hitems, (int)d->nhitems, g, d->hA, d->hB, d->part);
  PB_LAUNCHED("k_coef (half list)");
  PB_CUDA(cudaStreamSynchronize(st));  // host staging vectors are released on return
  return PB_OK;
}

template <typename IDX>
void set_stream_smem(int bytes) {
  cudaFuncSetAttribute(dev::k_stream_ff<dev::MODE_COLL, true, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(dev::k_stream_ff<dev::MODE_RATE, true, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(dev::k_stream_ff<dev::MODE_COLL, true, IDX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(dev::k_stream_ff<dev::MODE_RATE, true, IDX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(dev::k_stream_f64<dev::MODE_COLL, true, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(dev::k_stream_f64<dev::MODE_RATE, true, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

extern "C" int pb_dev_arena_bytes(const pb_channels *ch, const pb_dev_opts *opts, size_t *bytes) {
  clear_error();
  if (!ch || !bytes) return set_error(PB_EINVAL, "pb_dev_arena_bytes: null argument");
  int sm = 152;
  {
    int devid = 0;
    if (cudaGetDevice(&devid) == cudaSuccess) cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, devid);
    else cudaGetLastError();
  }
  pb_dev_opts o;
  int rc = resolve_opts(ch, opts, sm, o);
  if (rc) return rc;
  const bool c32 = o.variant == PB_VARIANT_C32;
  if (c32) o.variant = PB_VARIANT_FF;  // the FF device with FP32 tiles
  Plan P, S;
  try {
    bool complete = false;
    const bool merged = make_plans(ch, opts, o, sm, P, S, &complete);
    const int nfin = (int)((P.ns + kFinBlock - 1) / kFinBlock);
    const bool sym = sym_for(o, merged, complete, ch->closed, merged && tiles_pay(S.ns, S.nchp));
    if (c32 && !sym)
      return set_error(PB_EINVAL, "pb_dev: the FP32 coefficient tiles (C32) need the symmetric tiles: a "
                                  "closure-checked list whose rows are complete or miss few partners (or dense_rows 3)");
    const TrRows tr = tr_rows_for(P.ns, sm, o.transport != 0, merged, complete, o.variant, o);
    *bytes = make_layout(ch, P, merged ? &S : nullptr, o.variant, o.transport != 0, nfin, sym,
                         gdense_for(ch, o, sm), o.adjoint != 0, c32 ? sizeof(float2) : sizeof(float4), tr.nseg)
                 .total;
  } catch (const std::bad_alloc &) {
    return set_error(PB_ENOMEM, "pb_dev_arena_bytes: out of host memory");
  }
  return PB_OK;
}

namespace {
int coef_setup(pb_dev *d, cudaStream_t st);
}

extern "C" int pb_dev_create(const pb_channels *ch, const pb_dev_opts *opts, void *arena, size_t arena_bytes,
                             void *stream, pb_dev **out) {
  clear_error();
  if (!ch || !arena || !out) return set_error(PB_EINVAL, "pb_dev_create: null argument");
  *out = nullptr;
  if (((uintptr_t)arena) % kAlign) return set_error(PB_EINVAL, "pb_dev_create: arena must be 256-byte aligned");
  int sm = 0;
  int rc = check_device(&sm);
  if (rc) return rc;
  pb_dev_opts o;
  rc = resolve_opts(ch, opts, sm, o);
  if (rc) return rc;
  const bool c32 = o.variant == PB_VARIANT_C32;
  if (c32) o.variant = PB_VARIANT_FF;  // the FF device with FP32 tiles
  if (ch->nstate > INT32_MAX / 4) return set_error(PB_EINVAL, "pb_dev_create: too many states");
  cudaStream_t st = (cudaStream_t)stream;

  pb_dev *d = new (std::nothrow) pb_dev();
  if (!d) return set_error(PB_ENOMEM, "pb_dev_create: out of host memory");
  Plan P, S;
  bool merged = false, complete = false;
  try {
    merged = make_plans(ch, opts, o, sm, P, S, &complete);
  } catch (const std::bad_alloc &) {
    delete d;
    return set_error(PB_ENOMEM, "pb_dev_create: out of host memory");
  }
  const Plan &W = merged ? S : P;  // the sweep plan
  if (P.nitems > INT32_MAX || W.nitems > INT32_MAX) {
    delete d;
    return set_error(PB_EINVAL, "pb_dev_create: too many work items");
  }
  d->variant = o.variant;
  d->ns = ch->nstate;
  d->nch = ch->nch;
  d->nchp = P.nchp;
  d->nitems = W.nitems;
  d->merged = merged;
  d->ncitems = P.nitems;
  d->nsw = W.nchp;
  for (int i = 0; i < 3; ++i) d->nk[i] = ch->nk[i];
  d->nmodes = ch->nmodes;
  d->nq = ch->nq;
  d->T = ch->T;
  d->sigma = ch->sigma;
  d->c = 2.0 * kPi / (kHbar * (double)ch->nq);
  if (o.variant == PB_VARIANT_H16) {
    // FP16 |g|^2: the largest value at creation maps into [2^9, 2^10), so every value down to
    // 2^-23 of it stays a normal FP16 number (11 significand bits; FP16's smallest normal is
    // 2^-14) and pb_dev_set_g2 may raise them up to 63-fold
    double gmax = 0.0;
    for (const double v : ch->g2) gmax = std::max(gmax, std::fabs(v));
    if (gmax > 0.0 && std::isfinite(gmax)) d->g2s = std::ldexp(1.0, 10 - std::ilogb(gmax) - 1);
  }
  d->sm_count = sm;
  d->ctas = o.ctas_per_sm;
  d->item_ch = o.item_channels;
  d->transport = o.transport != 0;
  d->nfin_blocks = (int)((d->ns + kFinBlock - 1) / kFinBlock);
  d->sym = sym_for(o, merged, complete, ch->closed, merged && tiles_pay(S.ns, S.nchp));
  d->complete = complete;
  if (c32 && !d->sym) {
    delete d;
    return set_error(PB_EINVAL, "pb_dev: the FP32 coefficient tiles (C32) need the symmetric tiles: a "
                                "closure-checked list whose rows are complete or miss few partners (or dense_rows 3)");
  }
  d->c32 = c32;
  d->c32_shape = o.tile_sweep;
  d->sym_nt = d->sym && (o.tile_sweep == 2 || (o.tile_sweep == 3 && !c32)) ? dev::kSymThreads : 0;
  d->sym_half = d->sym && o.tile_sweep == 3 && !c32;
  d->half_cps = (opts && opts->ctas_per_sm == 2) ? 2 : 3;
  d->td = tile_dims(d->ns);
  const GDense gd = gdense_for(ch, o, sm);
  d->gdense = gd.on;
  d->gd_npp = gd.npp;
  d->gd_nitems = (int)gd.nitems;
  d->gd_bytes = gd.bytes;
  const TrRows trr = tr_rows_for(d->ns, sm, d->transport, merged, complete, o.variant, o);
  d->tr_nseg = trr.nseg;
  d->tr_seglen = trr.seglen;
  d->L = make_layout(ch, P, merged ? &S : nullptr, o.variant, d->transport, d->nfin_blocks, d->sym, gd,
                     o.adjoint != 0, c32 ? sizeof(float2) : sizeof(float4), trr.nseg);
  if (arena_bytes < d->L.total) {
    const size_t need = d->L.total;
    delete d;
    return set_error(PB_ENOMEM, "pb_dev_create: arena of %zu bytes is smaller than the %zu needed", arena_bytes, need);
  }
  d->arena = (char *)arena;
  d->arena_bytes = arena_bytes;
  char *A = d->arena;
  const Layout &L = d->L;
  d->rp = (int64_t *)(A + L.rp);
  d->item_ptr = (int32_t *)(A + L.item_ptr);
  d->items = (Item *)(A + L.items);
  d->col = (uint32_t *)(A + L.col);
  d->g2 = (double *)(A + L.g2);
  d->coefA = A + L.coefA;
  d->coefB = A + L.coefB;
  d->wt = (float2 *)(A + L.wt);
  d->eps = (double *)(A + L.eps);
  d->kc = (short4 *)(A + L.kc);
  d->R = (double *)(A + L.R);
  d->omega = (double *)(A + L.omega);
  d->tab = (double2 *)(A + L.tab);
  d->part = (Part4 *)(A + L.part);
  d->acc = (double *)(A + L.acc);
  d->y = (double *)(A + L.y);
  d->yff = (float2 *)(A + L.yff);
  d->fstage = (double *)(A + L.fstage);
  d->Fa = (double *)(A + L.Fa);
  d->Fb = (double *)(A + L.Fb);
  d->Fff = (float2 *)(A + L.Fff);
  d->tau = (double *)(A + L.tau);
  d->invtau = (double *)(A + L.invtau);
  d->red = (double2 *)(A + L.red);
  d->scal = (double *)(A + L.scal);
  d->obs = (double *)(A + L.obs);
  d->err = (int *)(A + L.err);
  d->g2lo = A + L.g2lo;
  if (d->gdense) {
    d->g2d = A + L.g2d;
    d->gd_items = (Item *)(A + L.gditems);
    d->gd_item_ptr = (int32_t *)(A + L.gdptr);
  }
  d->gstate = (uint4 *)(A + L.gstate);
  d->tab32 = (float2 *)(A + L.tab32);
  d->col16 = d->ns <= 65536 ? (uint16_t *)(A + L.col16) : nullptr;
  d->rp_real = (int64_t *)(A + L.rp_real);
  d->vjpG = (float2 *)(A + L.vjpG);
  if (d->tr_nseg) {
    d->trptr = (int32_t *)(A + L.trptr);
    d->trpart = (Part4 *)(A + L.trpart);
  }
  d->g2tab = (float4 *)(A + L.g2tab);
  if (d->mixed() && o.adjoint) d->gaccg = (double *)(A + L.gaccg);
  d->vecs = (double *)(A + L.vecs);
  d->hcol = (uint32_t *)(A + L.hcol);
  d->hg2 = (double *)(A + L.hg2);
  d->hA = (float2 *)(A + L.hA);
  d->hB = (float2 *)(A + L.hB);
  d->sc = (float2 *)(A + L.sc);
  d->entries = (int32_t *)(A + L.entries);
  d->hitems = (Item *)(A + L.hitems);
  d->titems = (Item *)(A + L.titems);
  d->t_item_ptr = (int32_t *)(A + L.t_item_ptr);
  if (merged) {
    d->citems = (Item *)(A + L.citems);
    d->citem_ptr = (int32_t *)(A + L.citem_ptr);
    d->cpart = (Part4 *)(A + L.cpart);
    d->ccoefA = A + L.ccoefA;
    d->ccoefB = A + L.ccoefB;
    d->sidx16 = d->ns <= 65536 ? (uint16_t *)(A + L.sidx16) : nullptr;
    d->sidx32 = d->ns <= 65536 ? nullptr : (uint32_t *)(A + L.sidx32);
    d->pcstart = (int64_t *)(A + L.pcstart);
    d->pcnt = (uint8_t *)(A + L.pcnt);
    d->srp = (int64_t *)(A + L.srp);
    d->gitems = (Item *)(A + L.gitems);
    if (d->variant == PB_VARIANT_FF && o.adjoint) d->gacc = (float4 *)(A + L.gacc);
    if (d->sym) {
      d->tiles = (int2 *)(A + L.tiles);
      d->tcoef = (float4 *)(A + L.tcoef);
      d->tc32 = (float2 *)(A + L.tcoef);
      d->tpart = (float4 *)(A + L.tpart);
    }
  } else {
    d->citems = d->items;
    d->citem_ptr = d->item_ptr;
    d->cpart = d->part;
    d->ccoefA = d->coefA;
    d->ccoefB = d->coefB;
    d->sidx16 = d->col16;
    d->sidx32 = d->col;
  }

  // shared-memory staging sizes
  int devid = 0, smem_optin = 0;
  cudaGetDevice(&devid);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, devid);
  const size_t ns8 = (size_t)((d->ns + kRowPad - 1) / kRowPad * kRowPad);  // zero-padded for complete rows
  size_t fbytes = d->variant == PB_VARIANT_F64 ? sizeof(double) * (size_t)d->ns : sizeof(float2) * ns8;
  if (d->mixed()) {
    fbytes = sizeof(uint4) * (size_t)d->ns;
    if (fbytes + 1024 > (size_t)smem_optin) {
      delete d;
      return set_error(PB_EINVAL, "pb_dev_create: the FP32/BF16/FP16 variants stage 16 bytes per state in shared memory; "
                                  "%lld states exceed it", (long long)ch->nstate);
    }
    for (int i = 0; i < 3; ++i) d->rad[i] = ch->nk[i] > 1 ? 2 * ch->nk[i] : 1;
    if ((double)d->rad[0] * d->rad[1] * d->rad[2] * ch->nmodes >= (double)(1 << dev::kRecLnmBits)) {
      delete d;
      return set_error(PB_EINVAL, "pb_dev_create: the FP32/BF16/FP16 variants need (2 N1)(2 N2)(2 N3) nmodes < 2^27 "
                                  "(padded phonon table index in the state records)");
    }
    d->ctas = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(228 * 1024) / (fbytes + 1024)));  // of 512 threads
  }
  const size_t per_cta_budget = (size_t)(228 * 1024) / (size_t)d->ctas - 1024;
  d->smem_f = (fbytes <= per_cta_budget && fbytes <= (size_t)smem_optin) ? fbytes : 0;
  if (d->mixed()) d->smem_f = fbytes;
  const size_t Fbytes = sizeof(float2) * 3 * ns8;
  const bool F_fits = Fbytes <= (size_t)smem_optin - 1024;
  // automatic: gather F through L1 (measured faster on GB300 than shared-memory staging,
  // which limits residency to one 512-thread CTA per SM at 40^3)
  d->smem_F = (o.transport_gather == 1 && F_fits) ? Fbytes : 0;
  d->tr_lane = o.transport_gather != 2;  // 2 = L1 gathers with 4-channel groups per lane
  // automatic: one 1024-thread CTA per SM with F in shared memory (0.259 ms per 40^3 iteration
  // on GB300 against 0.357 ms for 256-thread CTAs gathering F through L1)
  d->tr_shape = o.transport_gather == 0 ? 4 : o.transport_gather >= 3 ? o.transport_gather : 3;
  if (d->tr_shape == 4 && !F_fits) d->tr_shape = 5;
  d->smem_F1k = d->tr_shape == 4 ? Fbytes : 0;
  d->g_lane = o.channel_per_lane != 2;   // 2 = 4-channel groups per lane in the mixed-precision sweep
  // automatic: one 1024-thread CTA per SM with register prefetch (measured fastest on GB300
  // for both FP32 and BF16 |g|^2 at 40^3: 0.29 ms against 0.35-0.38 ms for the 512-thread shapes)
  d->g_shape = o.channel_per_lane == 0 ? 4 : o.channel_per_lane >= 3 ? o.channel_per_lane : 1;
  if (o.stream_mode == 2) {
    if (d->variant != PB_VARIANT_FF || d->ns > 65536) {
      delete d;
      return set_error(PB_EINVAL, "pb_dev_create: the bulk-copy sweep needs the FF variant and nstate <= 65536");
    }
    int cap = 8;
    for (const Item &it : W.items) cap = std::max(cap, it.len);
    const size_t fb = ((size_t)d->ns * sizeof(float2) + 127) / 128 * 128;
    const size_t sb = ((size_t)cap * (2 * sizeof(float2) + sizeof(uint16_t)) + 127) / 128 * 128;
    const size_t need = fb + dev::kBulkStages * sb + (dev::kBulkStages + 1) * 8 + dev::kBulkStages * sizeof(Item) +
                        2 * 32 * sizeof(double);
    if (need > (size_t)smem_optin) {
      delete d;
      return set_error(PB_EINVAL, "pb_dev_create: bulk-copy sweep needs %zu bytes of shared memory", need);
    }
    d->bulk = true;
    d->bulk_cap = cap;
    d->bulk_smem = need;
  }
  if (o.transport_gather == 1 && !F_fits) {
    delete d;
    return set_error(PB_EINVAL, "pb_dev_create: F of %lld states does not fit in shared memory", (long long)ch->nstate);
  }
  // complete rows: the FF sweeps take partners from entry positions (needs f in shared memory)
  d->dense = merged && complete && o.dense_rows != 2 && d->variant == PB_VARIANT_FF && d->smem_f && !d->bulk;
  // the row-block transport sweep (one CTA per SM, each partner's F read once for four rows):
  // measured slower than shape 4 on GB300 (64 against 57.8 us per 40^3 iteration), so only on request
  const bool rows_fit = d->tr_nseg && dev::tr_rows_smem((int)d->ns) <= (size_t)smem_optin;
  if (d->transport && d->dense && rows_fit && o.transport_gather == 7) {
    d->tr_shape = 7;
  } else if (d->transport && o.transport_gather == 7) {
    delete d;
    return set_error(PB_EINVAL, "pb_dev_create: transport_gather 7 needs complete, branch-merged float-float rows "
                                "whose F (24 bytes per state) and weight rings fit in shared memory");
  }
  d->smem_Frows = d->tr_shape == 7 ? dev::tr_rows_smem((int)d->ns) : 0;
  d->ctas_tr = d->smem_F ? (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(228 * 1024) / (d->smem_F + 1024))) : 8;
  if (o.transport_ctas > 0) d->ctas_tr = std::min(d->ctas_tr, o.transport_ctas);
  if (!d->smem_F && o.transport_ctas > 0) d->ctas_tr = o.transport_ctas;

  // host staging of the padded arrays
  int status = PB_OK;
  try {
    // rows in parallel (each writes only its own padded range; the arrays are filled, not
    // zeroed first)
    std::unique_ptr<uint32_t[]> colp(new uint32_t[(size_t)P.nchp]);
    std::unique_ptr<double[]> g2p(new double[(size_t)P.nchp]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < d->ns; ++r) {
      const int64_t a = ch->row_ptr[r], len = ch->row_ptr[r + 1] - a, b = P.rp[r], lenp = P.rp[r + 1] - b;
      for (int64_t i = 0; i < len; ++i) {
        colp[b + i] = (uint32_t)ch->col[a + i] | ((uint32_t)ch->nu[a + i] << kPartnerBits);
        g2p[b + i] = ch->g2[a + i];
      }
      for (int64_t i = len; i < lenp; ++i) {  // padding: self, branch 0, g2 = 0
        colp[b + i] = (uint32_t)r;
        g2p[b + i] = 0.0;
      }
    }
    std::vector<short4> kc((size_t)d->ns);
    const int N2 = ch->nk[1], N3 = ch->nk[2];
    for (int64_t r = 0; r < d->ns; ++r) {
      const int ik = ch->kidx[r];
      kc[r] = make_short4((short)(ik / (N2 * N3)), (short)((ik / N3) % N2), (short)(ik % N3), 0);
    }
    if (ch->nk[0] > 32767 || ch->nk[1] > 32767 || ch->nk[2] > 32767) {
      delete d;
      return set_error(PB_EINVAL, "pb_dev_create: grid dimension above 32767");
    }
#define UP(dst, src, bytes)                                                          \
  do {                                                                               \
    cudaError_t e_ = cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyHostToDevice, st); \
    if (e_ != cudaSuccess) {                                                         \
      status = cuda_fail(e_, "upload");                                              \
      break;                                                                         \
    }                                                                                \
  } while (0)
    do {
      {
        cudaError_t e_ = cudaMemsetAsync(d->err, 0, sizeof(int) * 4, st);
        if (e_ != cudaSuccess) {
          status = cuda_fail(e_, "clear error word");
          break;
        }
        // the tile sweeps copy the float-float f of a ragged last block rounded up to 16 bytes:
        // the padding after the nstate values must hold zeros (it multiplies zero coefficients)
        e_ = cudaMemsetAsync(d->yff, 0, align_up(sizeof(float2) * (size_t)d->ns), st);
        if (e_ != cudaSuccess) {
          status = cuda_fail(e_, "clear the stage input");
          break;
        }
      }
      UP(d->rp, P.rp.data(), sizeof(int64_t) * (d->ns + 1));
      if (d->gacc || d->gaccg) {
        cudaError_t e_ = d->gacc ? cudaMemsetAsync(d->gacc, 0, sizeof(float4) * (size_t)d->nsw, st)
                                 : cudaMemsetAsync(d->gaccg, 0, d->gaccg_bytes(), st);
        if (e_ != cudaSuccess) {
          status = cuda_fail(e_, "clear the gradient accumulators");
          break;
        }
      }
      if (d->gdense) {
        std::vector<int64_t> rpd((size_t)d->ns + 1);
        for (int64_t r = 0; r <= d->ns; ++r) rpd[r] = r * gd.npp;
        std::vector<Item> gi;
        std::vector<int32_t> gp;
        plan_items(rpd, gd.item, gi, gp);
        UP(d->gd_items, gi.data(), sizeof(Item) * gi.size());
        UP(d->gd_item_ptr, gp.data(), sizeof(int32_t) * gp.size());
      }
      if (d->tr_nseg) {  // the row-block transport sweep's partials: row r owns r * nseg .. (r + 1) * nseg
        std::vector<int32_t> tp((size_t)d->ns + 1);
        for (int64_t r = 0; r <= d->ns; ++r) tp[(size_t)r] = (int32_t)(r * d->tr_nseg);
        UP(d->trptr, tp.data(), sizeof(int32_t) * tp.size());
      }
      UP(d->rp_real, ch->row_ptr.data(), sizeof(int64_t) * (d->ns + 1));
      UP(d->item_ptr, W.item_ptr.data(), sizeof(int32_t) * (d->ns + 1));
      UP(d->items, W.items.data(), sizeof(Item) * W.nitems);
      if (merged) {
        UP(d->citem_ptr, P.item_ptr.data(), sizeof(int32_t) * (d->ns + 1));
        UP(d->citems, P.items.data(), sizeof(Item) * P.nitems);
      }
      UP(d->col, colp.get(), sizeof(uint32_t) * P.nchp);
      if (d->col16) {
        std::unique_ptr<uint16_t[]> c16(new uint16_t[(size_t)P.nchp]);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < P.nchp; ++i) c16[i] = (uint16_t)(colp[i] & kPartnerMask);
        UP(d->col16, c16.get(), sizeof(uint16_t) * P.nchp);  // pageable source: staged before return
      }
      UP(d->g2, g2p.get(), sizeof(double) * P.nchp);
      if (merged) {
        // one entry per run of equal partner in each row; padding entries: self, no channels
        std::unique_ptr<uint32_t[]> sidx(new uint32_t[(size_t)S.nchp]);
        std::unique_ptr<int64_t[]> cst(new int64_t[(size_t)S.nchp]);
        std::unique_ptr<uint8_t[]> cn(new uint8_t[(size_t)S.nchp]);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t r = 0; r < d->ns; ++r) {
          const int64_t a = ch->row_ptr[r], len = ch->row_ptr[r + 1] - a;
          int64_t e = S.rp[r];
          for (int64_t i = 0; i < len; ++i) {
            if (i > 0 && ch->col[a + i] == ch->col[a + i - 1]) {
              ++cn[e - 1];
              continue;
            }
            sidx[e] = (uint32_t)ch->col[a + i];
            cst[e] = P.rp[r] + i;
            cn[e] = 1;
            ++e;
          }
          for (; e < S.rp[r + 1]; ++e) {
            sidx[e] = (uint32_t)r;
            cst[e] = 0;
            cn[e] = 0;
          }
        }
        if (d->sidx16) {
          std::unique_ptr<uint16_t[]> s16(new uint16_t[(size_t)S.nchp]);
#pragma omp parallel for schedule(static)
          for (int64_t i = 0; i < S.nchp; ++i) s16[i] = (uint16_t)sidx[i];
          UP(d->sidx16, s16.get(), sizeof(uint16_t) * S.nchp);
        } else {
          UP(d->sidx32, sidx.get(), sizeof(uint32_t) * S.nchp);
        }
        UP(d->pcstart, cst.get(), sizeof(int64_t) * S.nchp);
        UP(d->pcnt, cn.get(), S.nchp);
        UP(d->srp, S.rp.data(), sizeof(int64_t) * (d->ns + 1));
        {
          std::vector<Item> gi;
          std::vector<int32_t> gptr;
          plan_items(S.rp, dev::kWarpChunk, gi, gptr);
          d->ngitems = (int)gi.size();
          UP(d->gitems, gi.data(), sizeof(Item) * gi.size());
        }
        if (d->sym) {
          std::vector<int2> tl;
          for (int I = 0; I < d->td.nb; ++I)
            for (int J = I; J < d->td.nb; ++J) tl.push_back(make_int2(I, J));
          UP(d->tiles, tl.data(), sizeof(int2) * tl.size());
          cudaError_t e2 = cudaStreamSynchronize(st);
          if (e2 != cudaSuccess) {
            status = cuda_fail(e2, "upload");
            break;
          }
        }
        cudaError_t e_ = cudaStreamSynchronize(st);  // pageable sources above go out of scope
        if (e_ != cudaSuccess) {
          status = cuda_fail(e_, "upload");
          break;
        }
      }
      UP(d->eps, ch->eps.data(), sizeof(double) * d->ns);
      UP(d->kc, kc.data(), sizeof(short4) * d->ns);
      UP(d->omega, ch->omega.data(), sizeof(double) * (size_t)ch->nq * ch->nmodes);
    } while (0);
#undef UP
    if (status == PB_OK) {
      const long long n = (long long)ch->nq * ch->nmodes;
      dev::k_table<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(d->omega, n, kBoltz * d->T, d->tab);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) status = cuda_fail(e, "k_table");
    }
    if (status == PB_OK) status = coef_setup(d, st);  // coefficients and R_s of the FF/F64 variants
    if (status == PB_OK && d->variant == PB_VARIANT_PAPER) status = paper_setup(d, ch, o.item_channels, st);
    if (status == PB_OK && d->mixed()) {
      dev::k_gstate_init<<<(int)((d->ns + 255) / 256), 256, 0, st>>>(d->eps, d->kc, (int)d->ns, d->rad[1], d->rad[2],
                                                                      ch->nmodes, d->gstate);
      const long long nt = (long long)d->rad[0] * d->rad[1] * d->rad[2] * ch->nmodes;
      dev::k_tab_padded<<<(int)std::min<long long>((nt + 255) / 256, 8192), 256, 0, st>>>(
          d->tab, ch->nk[0], ch->nk[1], ch->nk[2], d->rad[0], d->rad[1], d->rad[2], ch->nmodes, d->tab32);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) status = cuda_fail(e, "mixed-precision setup");
    }
    if (status == PB_OK) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) status = cuda_fail(e, "pb_dev_create: synchronize");
    }
  } catch (const std::bad_alloc &) {
    status = set_error(PB_ENOMEM, "pb_dev_create: out of host memory");
  }
  if (status != PB_OK) {
    delete d;
    return status;
  }
  if (d->bulk)
    cudaFuncSetAttribute(dev::k_stream_ff_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->bulk_smem);
  if (d->sym_nt) {
    if (dev::kSymBulkSmem > (size_t)smem_optin) {
      d->sym_nt = 0;  // the global-load tile sweep needs no opt-in shared memory
      d->sym_half = false;
    } else {
      cudaFuncSetAttribute(dev::k_stream_sym_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dev::kSymBulkSmem);
      cudaFuncSetAttribute(dev::k_stream_sym_half<3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)dev::half_smem<3>());
      cudaFuncSetAttribute(dev::k_stream_sym_half<2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)dev::half_smem<2>());
    }
  }
  if (d->c32)
    with_c32_shape(d->c32_shape, [&](auto nst, auto cps, auto half) {
      const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
      if constexpr (decltype(half)::value) {
        const int sm32 = (int)dev::c32_half_smem<nst()>();
        cudaFuncSetAttribute(dev::k_stream_c32_half<dev::MODE_COLL, nst(), cps()>, A, sm32);
        cudaFuncSetAttribute(dev::k_stream_c32_half<dev::MODE_RATE, nst(), cps()>, A, sm32);
      } else {
        const int sm32 = (int)dev::c32_smem<nst()>();
        cudaFuncSetAttribute(dev::k_stream_c32<dev::MODE_COLL, nst(), cps()>, A, sm32);
        cudaFuncSetAttribute(dev::k_stream_c32<dev::MODE_RATE, nst(), cps()>, A, sm32);
      }
    });
  if (d->smem_f > 48 * 1024) {
    set_stream_smem<uint32_t>((int)d->smem_f);
    set_stream_smem<uint16_t>((int)d->smem_f);
    cudaFuncSetAttribute(dev::k_paper_sc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem_f);
  }
  if (d->smem_F > 48 * 1024) {
    cudaFuncSetAttribute(dev::k_stream_tr<true, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem_F);
    cudaFuncSetAttribute(dev::k_stream_tr<true, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem_F);
  }
  if (d->smem_Frows > 48 * 1024)
    cudaFuncSetAttribute(dev::k_stream_tr_rows<dev::kTrRows>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)d->smem_Frows);
  if (d->smem_F1k > 48 * 1024) {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaFuncSetAttribute(dev::k_stream_tr_lane<uint32_t, 1024, true, true, true>, A, (int)d->smem_F1k);
    cudaFuncSetAttribute(dev::k_stream_tr_lane<uint16_t, 1024, true, true, true>, A, (int)d->smem_F1k);
    cudaFuncSetAttribute(dev::k_stream_tr_lane<uint32_t, 1024, true, true, true, true>, A, (int)d->smem_F1k);
    cudaFuncSetAttribute(dev::k_stream_tr_lane<uint16_t, 1024, true, true, true, true>, A, (int)d->smem_F1k);
  }
  {
    const size_t gb = sizeof(float2) * 3 * (size_t)d->ns;
    if (gb > 48 * 1024 && gb + 1024 <= (size_t)smem_optin) {
      cudaFuncSetAttribute(dev::k_stream_vjp<true, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gb);
      cudaFuncSetAttribute(dev::k_stream_vjp<true, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gb);
    }
    d->smem_G = gb + 1024 <= (size_t)smem_optin ? gb : 0;
  }
  if (d->mixed()) {
    const size_t vb = (sizeof(uint4) + sizeof(float)) * (size_t)d->ns;
    d->vjp_g_ok = vb + 1024 <= (size_t)smem_optin;
    if (vb > 48 * 1024 && d->vjp_g_ok)
      with_g2t(d->variant, [&](auto tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        cudaFuncSetAttribute(dev::k_stream_g_vjp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vb);
        cudaFuncSetAttribute(dev::k_stream_g_dense<dev::MODE_VJP, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vb);
      });
  }
  if (d->mixed() && d->smem_f > 48 * 1024)
    with_g2t(d->variant, [&](auto tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
      set_lane_smem<T>((int)d->smem_f);
      cudaFuncSetAttribute(dev::k_stream_g_dense<dev::MODE_COLL, T>, A, (int)d->smem_f);
      cudaFuncSetAttribute(dev::k_stream_g_dense<dev::MODE_RATE, T>, A, (int)d->smem_f);
      cudaFuncSetAttribute(dev::k_stream_g<dev::MODE_COLL, T>, A, (int)d->smem_f);
      cudaFuncSetAttribute(dev::k_stream_g<dev::MODE_RATE, T>, A, (int)d->smem_f);
    });
  cudaGetLastError();
  *out = d;
  return PB_OK;
}

extern "C" int pb_dev_check(pb_dev *d, void *stream) {
  clear_error();
  if (!d) return set_error(PB_EINVAL, "pb_dev_check: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  PB_CUDA(cudaMemcpyAsync(&h, d->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PB_CUDA(cudaStreamSynchronize(st));
  if (h) {
    PB_CUDA(cudaMemsetAsync(d->err, 0, sizeof(int), st));  // reported once
    PB_CUDA(cudaStreamSynchronize(st));
    if (h == dev::kErrG2Range)
      return set_error(PB_EINVAL, "a |g|^2 value overflowed the FP16 storage (more than 63 times the largest value "
                                  "at device creation)");
    if (h == dev::kErrG2Small)
      return set_error(PB_EINVAL, "a nonzero |g|^2 value is too small for the scaled FP16 storage (below 2^-23 of "
                                  "the largest value at device creation, it would keep fewer than 11 significand bits)");
    return set_error(PB_ETIMEOUT, "a bounded device-side wait gave up (error word %d)", h);
  }
  return PB_OK;
}

extern "C" int pb_dev_selftest_wait(pb_dev *d, int32_t wait_us, void *stream) {
  clear_error();
  if (!d) return set_error(PB_EINVAL, "pb_dev_selftest_wait: null argument");
  if (wait_us < 1 || wait_us > 2000000) return set_error(PB_EINVAL, "pb_dev_selftest_wait: wait_us must be 1..2000000");
  if (d->arena_bytes < 1024) return set_error(PB_EINVAL, "pb_dev_selftest_wait: the arena is smaller than the 1 KB copied");
  cudaStream_t st = (cudaStream_t)stream;
  dev::k_selftest_wait<<<1, 32, 0, st>>>((const float4 *)d->arena, 1000ull * (unsigned long long)wait_us, d->err);
  PB_LAUNCHED("k_selftest_wait");
  return PB_OK;
}

extern "C" void pb_dev_destroy(pb_dev *d) {
  if (!d) return;
  if (d->rk_exec) cudaGraphExecDestroy(d->rk_exec);
  if (d->rk_exec_in) cudaGraphExecDestroy(d->rk_exec_in);
  d->drop_call_graphs();
  if (d->cap) cudaStreamDestroy(d->cap);
  if (d->hres) cudaFreeHost(d->hres);
  for (cudaEvent_t e : d->hres_ev)
    if (e) cudaEventDestroy(e);
  delete d;
}

extern "C" int pb_dev_get_info(const pb_dev *d, pb_dev_info *info) {
  clear_error();
  if (!d || !info) return set_error(PB_EINVAL, "pb_dev_get_info: null argument");
  std::memset(info, 0, sizeof *info);
  info->nstate = d->ns;
  info->nchannels = d->nch;
  info->nchannels_padded = d->nchp;
  info->nitems = d->nitems;
  info->variant = d->c32 ? PB_VARIANT_C32 : d->variant;
  info->sm_count = d->sm_count;
  info->c = d->c;
  switch (d->variant) {
    // streamed bytes per physical channel: per sweep entry (state pair when branch-merged)
    case PB_VARIANT_FF:
      if (d->sym)
        info->bytes_per_channel = (double)(d->c32 ? sizeof(float2) : sizeof(float4)) * d->td.nt * dev::kTile *
                                  dev::kTile / (double)d->nch;
      else
        info->bytes_per_channel = (2 * sizeof(float2) + (d->dense ? 0 : d->sidx16 ? 2 : 4)) *
                                  (d->merged ? (double)d->nsw / (double)d->nch : 1.0);
      break;
    case PB_VARIANT_F64:
      info->bytes_per_channel = (2 * sizeof(double) + (d->sidx16 ? 2 : 4)) * (d->merged ? (double)d->nsw / (double)d->nch : 1.0);
      break;
    case PB_VARIANT_G32:
    case PB_VARIANT_G16:
    case PB_VARIANT_H16:
      // dense pair-major: the (state, partner, branch) slots, zeros included; else |g|^2 + word
      info->bytes_per_channel = d->gdense ? (d->nch ? (double)d->gd_bytes / (double)d->nch : 0.0)
                                          : (d->variant == PB_VARIANT_G32 ? 4.0 : 2.0) + sizeof(uint32_t);
      break;
    case PB_VARIANT_PAPER:  // step 2: P_in, D, index, sc_col write; step 3: entry + sc_col gather
      info->bytes_per_channel = d->nch ? (28.0 * (double)d->nh + 12.0 * (double)d->nent) / (double)d->nch : 0.0;
      break;
    default: info->bytes_per_channel = sizeof(double) + sizeof(uint32_t); break;
  }
  return PB_OK;
}

namespace {

// Stream pass over all items: part[item] = (A, B) or the literal sums.  `fd` is the
// distribution in double, `fff` its float-float copy (used by the FF variant); `colp` the
// partner indices (packed 32-bit words or the 16-bit copy).
template <typename IDX>
int launch_stream_t(pb_dev *d, int mode, const double *fd, const float2 *fff, const IDX *colp, Part4 *part,
                    cudaStream_t st) {
  const int grid = d->stream_grid(d->ctas);
  const int n = (int)d->nitems;
  const int ns = (int)d->ns;
  const bool coll = mode == dev::MODE_COLL;
  if (d->variant == PB_VARIANT_FF && coll && d->bulk) {
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>(d->nitems, (int64_t)d->sm_count));
    dev::k_stream_ff_bulk<<<gb, dev::kBlock, d->bulk_smem, st>>>(d->items, n, (const float2 *)d->coefA,
                                                                 (const float2 *)d->coefB, d->sidx16, fff, ns,
                                                                 d->bulk_cap, part, d->err);
  } else if (d->variant == PB_VARIANT_FF && d->sym && d->c32 && part == d->part && fff == d->yff) {
    // FP32 coefficient tiles through the bulk-copy ring (tiles32.cuh)
    float *tp = (float *)d->tpart;
    with_c32_shape(d->c32_shape, [&](auto nst, auto cps, auto half) {
      const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(d->td.nt, (int64_t)d->sm_count * cps()));
      if constexpr (decltype(half)::value) {
        const size_t sm32 = dev::c32_half_smem<nst()>();
        if (coll)
          dev::k_stream_c32_half<dev::MODE_COLL, nst(), cps()><<<gs, dev::kC32Threads, sm32, st>>>(
              d->tiles, d->td.nt, d->tc32, fff, ns, d->td.nb, tp, d->err, nullptr, d->rev);
        else
          dev::k_stream_c32_half<dev::MODE_RATE, nst(), cps()><<<gs, dev::kC32Threads, sm32, st>>>(
              d->tiles, d->td.nt, d->tc32, fff, ns, d->td.nb, tp, d->err, nullptr, d->rev);
      } else {
        const size_t sm32 = dev::c32_smem<nst()>();
        if (coll)
          dev::k_stream_c32<dev::MODE_COLL, nst(), cps()><<<gs, dev::kC32Threads, sm32, st>>>(
              d->tiles, d->td.nt, d->tc32, fff, ns, d->td.nb, tp, d->err, nullptr, d->rev);
        else
          dev::k_stream_c32<dev::MODE_RATE, nst(), cps()><<<gs, dev::kC32Threads, sm32, st>>>(
              d->tiles, d->td.nt, d->tc32, fff, ns, d->td.nb, tp, d->err, nullptr, d->rev);
      }
    });
  } else if (d->variant == PB_VARIANT_FF && d->sym && !d->c32 && part == d->part) {
    // symmetric tiles; the rate mode needs the same (A, B) partials
    if (d->sym_half && fff == d->yff) {
      const int cps = d->half_cps;
      const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(d->td.nt, (int64_t)d->sm_count * cps));
      if (cps == 3)
        dev::k_stream_sym_half<2, 3><<<gs, dev::kSymThreads, dev::half_smem<2>(), st>>>(
            d->tiles, d->td.nt, d->tcoef, fff, ns, d->td.nb, d->tpart, d->err, nullptr, d->rev);
      else
        dev::k_stream_sym_half<3, 2><<<gs, dev::kSymThreads, dev::half_smem<3>(), st>>>(
            d->tiles, d->td.nt, d->tcoef, fff, ns, d->td.nb, d->tpart, d->err, nullptr, d->rev);
    } else if (d->sym_nt && fff == d->yff) {  // the bulk copies read f from this padded arena buffer
      const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(d->td.nt, (int64_t)d->sm_count));
      dev::k_stream_sym_bulk<<<gs, dev::kSymThreads, dev::kSymBulkSmem, st>>>(d->tiles, d->td.nt, d->tcoef, fff, ns,
                                                                              d->td.nb, d->tpart, d->err);
    } else {
      const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(d->td.nt, (int64_t)d->sm_count * 3));
      dev::k_stream_sym<<<gs, 256, 0, st>>>(d->tiles, d->td.nt, d->tcoef, fff, ns, d->td.nb, d->tpart);
    }
  } else if (d->variant == PB_VARIANT_FF) {
    const float4 *A4 = (const float4 *)d->coefA, *B4 = (const float4 *)d->coefB;
    const long long *srp = (const long long *)d->srp;
    if (d->dense) {
      if (coll) dev::k_stream_ff<dev::MODE_COLL, true, IDX, true><<<grid, dev::kBlock, d->smem_f, st>>>(d->items, n, A4, B4, colp, fff, ns, part, srp);
      else      dev::k_stream_ff<dev::MODE_RATE, true, IDX, true><<<grid, dev::kBlock, d->smem_f, st>>>(d->items, n, A4, B4, colp, fff, ns, part, srp);
    } else if (d->smem_f) {
      if (coll) dev::k_stream_ff<dev::MODE_COLL, true, IDX><<<grid, dev::kBlock, d->smem_f, st>>>(d->items, n, A4, B4, colp, fff, ns, part);
      else      dev::k_stream_ff<dev::MODE_RATE, true, IDX><<<grid, dev::kBlock, d->smem_f, st>>>(d->items, n, A4, B4, colp, fff, ns, part);
    } else {
      if (coll) dev::k_stream_ff<dev::MODE_COLL, false, IDX><<<grid, dev::kBlock, 0, st>>>(d->items, n, A4, B4, colp, fff, ns, part);
      else      dev::k_stream_ff<dev::MODE_RATE, false, IDX><<<grid, dev::kBlock, 0, st>>>(d->items, n, A4, B4, colp, fff, ns, part);
    }
  } else if (d->variant == PB_VARIANT_F64) {
    const double2 *A2 = (const double2 *)d->coefA, *B2 = (const double2 *)d->coefB;
    if (d->smem_f) {
      if (coll) dev::k_stream_f64<dev::MODE_COLL, true, IDX><<<grid, dev::kBlock, d->smem_f, st>>>(d->items, n, A2, B2, colp, fd, ns, part);
      else      dev::k_stream_f64<dev::MODE_RATE, true, IDX><<<grid, dev::kBlock, d->smem_f, st>>>(d->items, n, A2, B2, colp, fd, ns, part);
    } else {
      if (coll) dev::k_stream_f64<dev::MODE_COLL, false, IDX><<<grid, dev::kBlock, 0, st>>>(d->items, n, A2, B2, colp, fd, ns, part);
      else      dev::k_stream_f64<dev::MODE_RATE, false, IDX><<<grid, dev::kBlock, 0, st>>>(d->items, n, A2, B2, colp, fd, ns, part);
    }
  } else if (d->variant == PB_VARIANT_PAPER) {
    if (!coll) return set_error(PB_EINVAL, "scattering rates are not available in the paper layout");
    const int64_t nh32 = (d->nhitems * 32 + dev::kBlock - 1) / dev::kBlock;
    const int gh = (int)std::max<int64_t>(1, std::min<int64_t>(nh32, (int64_t)d->sm_count * d->ctas));
    const float4 *A4 = (const float4 *)d->hA, *B4 = (const float4 *)d->hB;
    if (d->smem_f)
      dev::k_paper_sc<true><<<gh, dev::kBlock, d->smem_f, st>>>(d->hitems, (int)d->nhitems, A4, B4, d->hcol, fff, ns, (float4 *)d->sc);
    else
      dev::k_paper_sc<false><<<gh, dev::kBlock, 0, st>>>(d->hitems, (int)d->nhitems, A4, B4, d->hcol, fff, ns, (float4 *)d->sc);
    PB_LAUNCHED("k_paper_sc");
    const int64_t nt32 = (d->ntitems * 32 + dev::kBlock - 1) / dev::kBlock;
    const int gt = (int)std::max<int64_t>(1, std::min<int64_t>(nt32, (int64_t)d->sm_count * 4));
    dev::k_paper_gather<<<gt, dev::kBlock, 0, st>>>(d->titems, (int)d->ntitems, d->entries, d->sc, part);
  } else if (d->mixed()) {
    const dev::GGeom g = d->ggeom();
    const int gg = (int)std::max<int64_t>(1, std::min<int64_t>((d->nitems * 32 + 511) / 512, (int64_t)d->sm_count * d->ctas));
    with_g2t(d->variant, [&](auto tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      const T *gl = (const T *)d->g2lo;
      if (d->gdense) {
        const int gdg = (int)std::max<int64_t>(
            1, std::min<int64_t>(((int64_t)d->gd_nitems * 32 + dev::kDenseThreads - 1) / dev::kDenseThreads, d->sm_count));
        const int nd = d->gd_nitems, npp = d->gd_npp, nm = d->nmodes;
        const T *gd = (const T *)d->g2d;
        if (coll) dev::k_stream_g_dense<dev::MODE_COLL, T><<<gdg, dev::kDenseThreads, d->smem_f, st>>>(d->gd_items, nd, g, gd, npp, nm, d->gstate, ns, part);
        else      dev::k_stream_g_dense<dev::MODE_RATE, T><<<gdg, dev::kDenseThreads, d->smem_f, st>>>(d->gd_items, nd, g, gd, npp, nm, d->gstate, ns, part);
      } else if (d->g_lane) {
        launch_g_lane<T>(d->g_shape, coll, gg, d->sm_count, d->smem_f, st, d->items, n, g, gl, d->gstate, ns, part);
      } else {
        if (coll) dev::k_stream_g<dev::MODE_COLL, T><<<gg, 512, d->smem_f, st>>>(d->items, n, g, gl, d->gstate, ns, part);
        else      dev::k_stream_g<dev::MODE_RATE, T><<<gg, 512, d->smem_f, st>>>(d->items, n, g, gl, d->gstate, ns, part);
      }
    });
  } else {
    const dev::ChanGeom g = d->geom();
    const int lgrid = d->stream_grid(8);
    if (coll) dev::k_stream_literal<dev::MODE_COLL><<<lgrid, dev::kBlock, 0, st>>>(d->items, n, g, fd, part);
    else      dev::k_stream_literal<dev::MODE_RATE><<<lgrid, dev::kBlock, 0, st>>>(d->items, n, g, fd, part);
  }
  PB_LAUNCHED("stream kernel");
  return PB_OK;
}

int launch_stream_to(pb_dev *d, int mode, const double *fd, const float2 *fff, Part4 *part, cudaStream_t st) {
  if (d->sidx16) return launch_stream_t<uint16_t>(d, mode, fd, fff, d->sidx16, part, st);
  return launch_stream_t<uint32_t>(d, mode, fd, fff, d->sidx32, part, st);
}

int launch_stream(pb_dev *d, int mode, const double *fd, const float2 *fff, cudaStream_t st) {
  return launch_stream_to(d, mode, fd, fff, d->part, st);
}

int fin_grid(const pb_dev *d) { return d->nfin_blocks; }

// the tile epilogues: 8 states per CTA unless 32 per CTA still give four CTAs per SM (with 32
// per CTA a 40^3 step had 149 CTAs for 152 SMs, and the C32 RK4 step ran 14% slower)
bool fin_small(const pb_dev *d) { return (d->ns + 31) / 32 < 4 * (int64_t)d->sm_count; }

// ydst: where a stage writes the next stage's input (default d->y)
template <int STAGE>
void launch_fin(pb_dev *d, const double *ysrc, double *out, double *f, double dt, cudaStream_t st,
                double *ydst = nullptr) {
  double *y = ydst ? ydst : d->y;
  if (d->mixed())
    dev::k_fin_coll<true, STAGE, true><<<fin_grid(d), kFinBlock, 0, st>>>(dev::ItemSrc{d->fwd_item_ptr(), d->part}, (int)d->ns,
                                                                          d->gscale(), d->R,
                                                                          ysrc, out, f, d->acc, y,
                                                                          (float2 *)d->gstate, dt);
  else if (d->variant == PB_VARIANT_LITERAL || d->variant == PB_VARIANT_PAPER)
    dev::k_fin_coll<true, STAGE><<<fin_grid(d), kFinBlock, 0, st>>>(
        dev::ItemSrc{d->variant == PB_VARIANT_PAPER ? d->t_item_ptr : d->item_ptr, d->part}, (int)d->ns, d->c, d->R, ysrc,
                                                                    out, f, d->acc, y, d->yff, dt);
  else if (d->sym && d->c32)
    if (fin_small(d))
      dev::k_fin_c32<STAGE, false, 8><<<(int)((d->ns + 7) / 8), 256, 0, st>>>(
          (const float *)d->tpart, d->td.nb, d->td.nsp, (int)d->ns, d->c, ysrc, out, f, d->acc, y, d->yff, dt);
    else
      dev::k_fin_c32<STAGE><<<(int)((d->ns + 31) / 32), 256, 0, st>>>(
          (const float *)d->tpart, d->td.nb, d->td.nsp, (int)d->ns, d->c, ysrc, out, f, d->acc, y, d->yff, dt);
  else if (d->sym)
    if (fin_small(d))
      dev::k_fin_tiles<STAGE, false, 8><<<(int)((d->ns + 7) / 8), 256, 0, st>>>(
          dev::TileSrc{d->tpart, d->td.nb, d->td.nsp}, (int)d->ns, d->c, d->R, ysrc, out, f, d->acc, y, d->yff, dt);
    else
      dev::k_fin_tiles<STAGE><<<(int)((d->ns + 31) / 32), 256, 0, st>>>(
          dev::TileSrc{d->tpart, d->td.nb, d->td.nsp}, (int)d->ns, d->c, d->R, ysrc, out, f, d->acc, y, d->yff, dt);
  else
    dev::k_fin_coll<false, STAGE><<<fin_grid(d), kFinBlock, 0, st>>>(dev::ItemSrc{d->item_ptr, d->part}, (int)d->ns, d->c, d->R, ysrc,
                                                                     out, f, d->acc, y, d->yff, dt);
}

int to_ff(pb_dev *d, const double *x, int64_t n, float2 *out, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024));
  dev::k_to_ff<<<grid, 256, 0, st>>>(x, (long long)n, out);
  PB_LAUNCHED("k_to_ff");
  return PB_OK;
}

// Stage-input conversion the streaming kernel of this variant reads (once per call: splitting
// f inside every CTA of the sweep instead costs more, FP64 being slow on this part).
int stage_input(pb_dev *d, const double *f, cudaStream_t st) {
  if (d->variant == PB_VARIANT_FF || d->variant == PB_VARIANT_PAPER) return to_ff(d, f, d->ns, d->yff, st);
  if (d->mixed()) {
    dev::k_gstate_f<<<(int)((d->ns + 255) / 256), 256, 0, st>>>(f, (int)d->ns, d->gstate);
    PB_LAUNCHED("k_gstate_f");
  }
  return PB_OK;
}

// One RK4 step on the device vector f (the stage-0 ff copy must already be in yff).
// the four stages; the tile sweeps of stages 2 and 4 take the tile list from its end, so that
// each starts on the tiles the sweep before it left in L2 (and the next step's first sweep on
// those of the fourth)
int rk4_stages(pb_dev *d, double *f, double dt, cudaStream_t st) {
  int rc;
  d->rev = 0;
  if ((rc = launch_stream(d, dev::MODE_COLL, f, d->yff, st))) return rc;
  launch_fin<0>(d, f, nullptr, f, dt, st);
  PB_LAUNCHED("rk4 stage 1");
  d->rev = 1;
  if ((rc = launch_stream(d, dev::MODE_COLL, d->y, d->yff, st))) return rc;
  launch_fin<1>(d, d->y, nullptr, f, dt, st);
  PB_LAUNCHED("rk4 stage 2");
  d->rev = 0;
  if ((rc = launch_stream(d, dev::MODE_COLL, d->y, d->yff, st))) return rc;
  launch_fin<2>(d, d->y, nullptr, f, dt, st);
  PB_LAUNCHED("rk4 stage 3");
  d->rev = 1;
  if ((rc = launch_stream(d, dev::MODE_COLL, d->y, d->yff, st))) return rc;
  launch_fin<3>(d, d->y, nullptr, f, dt, st);
  PB_LAUNCHED("rk4 stage 4");
  return PB_OK;
}

int rk4_launches(pb_dev *d, double *f, double dt, cudaStream_t st) {
  const int rc = rk4_stages(d, f, dt, st);
  d->rev = 0;
  return rc;
}

void drop_rk_graphs(pb_dev *d) {
  if (d->rk_exec) cudaGraphExecDestroy(d->rk_exec);
  if (d->rk_exec_in) cudaGraphExecDestroy(d->rk_exec_in);
  d->rk_exec = d->rk_exec_in = nullptr;
}

// two graphs of one RK4 step on f: rk_exec (its stage input already in yff, as the last stage
// of a step leaves it) and rk_exec_in (the conversion of f first, for a call's first step)
int ensure_rk_graph(pb_dev *d, double *f, double dt) {
  if (d->rk_exec && d->rk_exec_in && d->rk_f == f && d->rk_dt == dt) return PB_OK;
  drop_rk_graphs(d);
  if (!d->cap) PB_CUDA(cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking));
  for (int with_input = 0; with_input < 2; ++with_input) {
    PB_CUDA(cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeThreadLocal));
    int rc = with_input ? stage_input(d, f, d->cap) : PB_OK;
    if (rc == PB_OK) rc = rk4_launches(d, f, dt, d->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(d->cap, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      drop_rk_graphs(d);
      return rc;
    }
    if (e != cudaSuccess) {
      drop_rk_graphs(d);
      return cuda_fail(e, "cudaStreamEndCapture");
    }
    cudaGraphExec_t &exec = with_input ? d->rk_exec_in : d->rk_exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      exec = nullptr;
      drop_rk_graphs(d);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  d->rk_f = f;
  d->rk_dt = dt;
  return PB_OK;
}

int ensure_weights(pb_dev *d, const double *f0, cudaStream_t st) {
  if (!d->transport) return set_error(PB_EINVAL, "transport buffers were not reserved (pb_dev_opts.transport = 0)");
  const int grid = d->stream_grid(8);
  if (d->variant == PB_VARIANT_FF || d->variant == PB_VARIANT_F64) {
    // from the coefficient arrays (per state pair when branch-merged)
    const bool ff = d->variant == PB_VARIANT_FF;
    const int n = (int)d->nitems;
    if (d->sidx16) {
      if (ff) dev::k_weights_coef<true, uint16_t><<<grid, dev::kBlock, 0, st>>>(d->items, n, d->coefA, d->coefB, d->sidx16, f0, d->c, d->wt, d->part);
      else    dev::k_weights_coef<false, uint16_t><<<grid, dev::kBlock, 0, st>>>(d->items, n, d->coefA, d->coefB, d->sidx16, f0, d->c, d->wt, d->part);
    } else {
      if (ff) dev::k_weights_coef<true, uint32_t><<<grid, dev::kBlock, 0, st>>>(d->items, n, d->coefA, d->coefB, d->sidx32, f0, d->c, d->wt, d->part);
      else    dev::k_weights_coef<false, uint32_t><<<grid, dev::kBlock, 0, st>>>(d->items, n, d->coefA, d->coefB, d->sidx32, f0, d->c, d->wt, d->part);
    }
  } else {
    dev::k_weights<<<grid, dev::kBlock, 0, st>>>(d->items, (int)d->nitems, d->geom(), f0, d->c, d->wt, d->part);
  }
  PB_LAUNCHED("k_weights");
  dev::k_rowsum<<<(int)((d->ns + 255) / 256), 256, 0, st>>>(d->item_ptr, d->part, (int)d->ns, d->invtau);
  PB_LAUNCHED("k_rowsum");
  dev::k_recip<<<(int)((d->ns + 255) / 256), 256, 0, st>>>(d->invtau, (int)d->ns, d->tau);
  PB_LAUNCHED("k_recip");
  return PB_OK;
}

// Lane-mapped transport sweep shapes (pb_dev_opts.transport_gather): 3 = 256-thread CTAs,
// F through L1; 4 = one 1024-thread CTA per SM, F in shared memory, next trip in registers,
// lazily renormalised float-float sums; 5 = the same with F through L1; 6 = shape 3 with the
// lazy sums.
template <typename IDX>
void launch_tr_lane(pb_dev *d, const IDX *col, const float2 *Fin, cudaStream_t st) {
  using namespace pb::dev;
  const int n = (int)d->nitems, ns = (int)d->ns;
  const int64_t need = (d->nitems * 32 + kBlock - 1) / kBlock;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)d->sm_count * d->ctas_tr));
  const int grid1k = (int)std::max<int64_t>(1, std::min<int64_t>((d->nitems * 32 + 1023) / 1024, d->sm_count));
  switch (d->tr_shape) {
    case 4:
      if (d->dense)
        k_stream_tr_lane<IDX, 1024, true, true, true, true><<<grid1k, 1024, d->smem_F1k, st>>>(
            d->items, n, d->wt, col, Fin, ns, d->part, (const long long *)d->srp);
      else
        k_stream_tr_lane<IDX, 1024, true, true, true><<<grid1k, 1024, d->smem_F1k, st>>>(d->items, n, d->wt, col, Fin, ns, d->part);
      break;
    case 5:
      k_stream_tr_lane<IDX, 1024, false, true, true><<<grid1k, 1024, 0, st>>>(d->items, n, d->wt, col, Fin, ns, d->part);
      break;
    case 6:
      k_stream_tr_lane<IDX, kBlock, false, false, true><<<grid, kBlock, 0, st>>>(d->items, n, d->wt, col, Fin, ns, d->part);
      break;
    default:
      k_stream_tr_lane<IDX, kBlock, false, false, false><<<grid, kBlock, 0, st>>>(d->items, n, d->wt, col, Fin, ns, d->part);
  }
}

// res3: where the residual numbers go (d->scal when null)
int transport_pass(pb_dev *d, const float2 *Fin_ff, const double *vel3, const double *Fold, double *Fnew,
                   float2 *Fnew_ff, cudaStream_t st, double *res3 = nullptr) {
  const int n = (int)d->nitems;
  const float4 *W4 = (const float4 *)d->wt;
  const int64_t need = (d->nitems * 32 + dev::kBlock - 1) / dev::kBlock;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)d->sm_count * d->ctas_tr));
  const bool rows = d->tr_shape == 7;
  if (rows) {
    const int64_t nit = (d->ns + dev::kTrRows - 1) / dev::kTrRows * (int64_t)d->tr_nseg;
    constexpr int wpc = dev::kTrThreads / 32;
    const int gr = (int)std::max<int64_t>(1, std::min<int64_t>((nit + wpc - 1) / wpc, d->sm_count));
    dev::k_stream_tr_rows<dev::kTrRows><<<gr, dev::kTrThreads, d->smem_Frows, st>>>(
        d->wt, (const long long *)d->srp, Fin_ff, (int)d->ns, d->tr_nseg, d->tr_seglen, d->trpart);
  } else if (d->smem_F) {
    if (d->sidx16) dev::k_stream_tr<true, uint16_t><<<grid, dev::kBlock, d->smem_F, st>>>(d->items, n, W4, d->sidx16, Fin_ff, (int)d->ns, d->part);
    else           dev::k_stream_tr<true, uint32_t><<<grid, dev::kBlock, d->smem_F, st>>>(d->items, n, W4, d->sidx32, Fin_ff, (int)d->ns, d->part);
  } else if (d->tr_lane) {
    if (d->sidx16) launch_tr_lane<uint16_t>(d, d->sidx16, Fin_ff, st);
    else           launch_tr_lane<uint32_t>(d, d->sidx32, Fin_ff, st);
  } else {
    if (d->sidx16) dev::k_stream_tr<false, uint16_t><<<grid, dev::kBlock, 0, st>>>(d->items, n, W4, d->sidx16, Fin_ff, (int)d->ns, d->part);
    else           dev::k_stream_tr<false, uint32_t><<<grid, dev::kBlock, 0, st>>>(d->items, n, W4, d->sidx32, Fin_ff, (int)d->ns, d->part);
  }
  PB_LAUNCHED("k_stream_tr");
  dev::k_fin_tr<<<fin_grid(d), kFinBlock, 0, st>>>(rows ? d->trptr : d->item_ptr, rows ? d->trpart : d->part,
                                                    (int)d->ns, d->tau, vel3, Fold, Fnew, Fnew_ff, d->red);
  PB_LAUNCHED("k_fin_tr");
  dev::k_red_final<<<1, 256, 0, st>>>(d->red, d->nfin_blocks, res3 ? res3 : d->scal);
  PB_LAUNCHED("k_red_final");
  return PB_OK;
}

}  // namespace

namespace {
// Runs the launch sequence `seq(stream)` of a call from a CUDA graph kept for this call kind and
// argument set (captured on first use; the last pb_dev::kGraphs kept, the oldest replaced).  When
// `st` is itself being captured, the launches are recorded into the caller's capture instead.
template <typename Seq>
int replay(pb_dev *d, int kind, const void *a, const void *b, const void *c, const void *e, cudaStream_t st,
           Seq &&seq) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  PB_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return seq(st);
  cudaGraphExec_t exec = nullptr;
  for (auto &g : d->cg)
    if (g.exec && g.kind == kind && g.a == a && g.b == b && g.c == c && g.e == e) exec = g.exec;
  if (!exec) {
    if (!d->cap) PB_CUDA(cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking));
    PB_CUDA(cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeThreadLocal));
    const int rc = seq(d->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaStreamEndCapture(d->cap, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (err != cudaSuccess) return cuda_fail(err, "cudaStreamEndCapture");
    auto &g = d->cg[d->cg_next];
    d->cg_next = (d->cg_next + 1) % pb_dev::kGraphs;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = pb_dev::CallGraph{};
    err = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
      g.exec = nullptr;
      return cuda_fail(err, "cudaGraphInstantiate");
    }
    g.kind = kind;
    g.a = a;
    g.b = b;
    g.c = c;
    g.e = e;
    exec = g.exec;
  }
  PB_CUDA(cudaGraphLaunch(exec, st));
  return PB_OK;
}

enum { kCallCollision = 1, kCallRates = 2, kCallTransport = 3, kCallRk4Host = 4, kCallTransportHost = 5,
       kCallVjp = 6, kCallVjpDefer = 7, kCallSolvePass = 8 };

// page-locked host memory (pinned or registered), which a graph's copy nodes may address
bool pinned_host(const void *p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// one transport pass: conversion of F3in, sweep, epilogue, residual (into res3, or the handle's
// scalars when null)
int transport_seq(pb_dev *d, const double *vel3, const double *F3in, double *F3out, double *res3, cudaStream_t st) {
  int rc;
  if ((rc = to_ff(d, F3in, 3 * d->ns, d->Fff, st))) return rc;
  return transport_pass(d, d->Fff, vel3, F3in, F3out, d->Fff, st, res3);
}
}  // namespace

extern "C" int pb_collision(pb_dev *d, const double *f, double *dfdt, void *stream) {
  clear_error();
  if (!d || !f || !dfdt) return set_error(PB_EINVAL, "pb_collision: null argument");
  return replay(d, kCallCollision, f, dfdt, nullptr, nullptr, (cudaStream_t)stream, [&](cudaStream_t st) -> int {
    int rc;
    if ((rc = stage_input(d, f, st))) return rc;
    if ((rc = launch_stream(d, dev::MODE_COLL, f, d->yff, st))) return rc;
    launch_fin<-1>(d, f, dfdt, nullptr, 0.0, st);
    PB_LAUNCHED("k_fin_coll");
    return PB_OK;
  });
}

extern "C" int pb_dev_time_sweep(pb_dev *d, const double *f, int32_t nlaunch, int32_t order, float *avg_ms,
                                 void *stream) {
  clear_error();
  if (!d || !f || !avg_ms) return set_error(PB_EINVAL, "pb_dev_time_sweep: null argument");
  if (nlaunch < 1 || nlaunch > 10000) return set_error(PB_EINVAL, "pb_dev_time_sweep: nlaunch must be 1..10000");
  if (order < 0 || order > 1) return set_error(PB_EINVAL, "pb_dev_time_sweep: order must be 0 or 1");
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if ((rc = stage_input(d, f, st))) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PB_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(PB_ECUDA, "pb_dev_time_sweep: cudaEventCreate");
  }
  cudaError_t e = cudaEventRecord(e0, st);
  for (int i = 0; i < nlaunch && e == cudaSuccess && rc == PB_OK; ++i) {
    d->rev = order == 1 ? (i & 1) : 0;
    rc = launch_stream(d, dev::MODE_COLL, f, d->yff, st);
  }
  d->rev = 0;
  if (e == cudaSuccess && rc == PB_OK) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess && rc == PB_OK) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess && rc == PB_OK) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "pb_dev_time_sweep");
  *avg_ms = ms / (float)nlaunch;
  return PB_OK;
}

namespace {
int rates_seq(pb_dev *d, const double *f, double *inv_tau, cudaStream_t st);
}

extern "C" int pb_scatter_rates(pb_dev *d, const double *f, double *inv_tau, void *stream) {
  clear_error();
  if (!d || !f || !inv_tau) return set_error(PB_EINVAL, "pb_scatter_rates: null argument");
  if (d->variant == PB_VARIANT_PAPER)
    return set_error(PB_EINVAL, "scattering rates are not available in the paper layout");
  return replay(d, kCallRates, f, inv_tau, nullptr, nullptr, (cudaStream_t)stream,
                [&](cudaStream_t st) { return rates_seq(d, f, inv_tau, st); });
}

namespace {
int rates_seq(pb_dev *d, const double *f, double *inv_tau, cudaStream_t st) {
  int rc;
  if ((rc = stage_input(d, f, st))) return rc;
  if ((rc = launch_stream(d, dev::MODE_RATE, f, d->yff, st))) return rc;
  if (d->variant == PB_VARIANT_LITERAL || d->mixed())
    dev::k_fin_rate<true><<<fin_grid(d), kFinBlock, 0, st>>>(dev::ItemSrc{d->fwd_item_ptr(), d->part}, (int)d->ns,
                                                             d->mixed() ? d->gscale() : d->c, d->R, inv_tau);
  else if (d->sym && d->c32 && fin_small(d))
    dev::k_fin_c32<-1, true, 8><<<(int)((d->ns + 7) / 8), 256, 0, st>>>((const float *)d->tpart, d->td.nb, d->td.nsp,
                                                                       (int)d->ns, d->c, nullptr, inv_tau, nullptr,
                                                                       nullptr, nullptr, nullptr, 0.0);
  else if (d->sym && d->c32)
    dev::k_fin_c32<-1, true><<<(int)((d->ns + 31) / 32), 256, 0, st>>>((const float *)d->tpart, d->td.nb, d->td.nsp,
                                                                       (int)d->ns, d->c, nullptr, inv_tau, nullptr,
                                                                       nullptr, nullptr, nullptr, 0.0);
  else if (d->sym && fin_small(d))
    dev::k_fin_tiles<-1, true, 8><<<(int)((d->ns + 7) / 8), 256, 0, st>>>(
        dev::TileSrc{d->tpart, d->td.nb, d->td.nsp}, (int)d->ns, d->c, d->R, nullptr, inv_tau, nullptr, nullptr, nullptr,
        nullptr, 0.0);
  else if (d->sym)
    dev::k_fin_tiles<-1, true><<<(int)((d->ns + 31) / 32), 256, 0, st>>>(
        dev::TileSrc{d->tpart, d->td.nb, d->td.nsp}, (int)d->ns, d->c, d->R, nullptr, inv_tau, nullptr, nullptr, nullptr,
        nullptr, 0.0);
  else
    dev::k_fin_rate<false><<<fin_grid(d), kFinBlock, 0, st>>>(dev::ItemSrc{d->item_ptr, d->part}, (int)d->ns, d->c, d->R, inv_tau);
  PB_LAUNCHED("k_fin_rate");
  return PB_OK;
}
}  // namespace

extern "C" int pb_rtbte_rk4_step(pb_dev *d, double *f, double dt, int32_t nsteps, void *stream) {
  clear_error();
  if (!d || !f) return set_error(PB_EINVAL, "pb_rtbte_rk4_step: null argument");
  if (nsteps < 0 || !std::isfinite(dt)) return set_error(PB_EINVAL, "pb_rtbte_rk4_step: bad dt or nsteps");
  if (nsteps == 0) return PB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_rk_graph(d, f, dt);
  if (rc) return rc;
  PB_CUDA(cudaGraphLaunch(d->rk_exec_in, st));  // the first step converts f itself
  for (int32_t i = 1; i < nsteps; ++i) PB_CUDA(cudaGraphLaunch(d->rk_exec, st));
  return PB_OK;
}

extern "C" int pb_rtbte_rk4_host(pb_dev *d, const double *f_host_in, double *f_host_out, double dt, int32_t nsteps,
                                 void *stream) {
  clear_error();
  if (!d || !f_host_in || !f_host_out) return set_error(PB_EINVAL, "pb_rtbte_rk4_host: null argument");
  if (nsteps < 0 || !std::isfinite(dt)) return set_error(PB_EINVAL, "pb_rtbte_rk4_host: bad dt or nsteps");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * (size_t)d->ns;
  if (nsteps == 1 && pinned_host(f_host_in) && pinned_host(f_host_out)) {
    // one step from page-locked buffers: both copies and the step's launches in one graph,
    // replayed per (buffers, dt)
    uint64_t dtk = 0;
    std::memcpy(&dtk, &dt, sizeof dtk);
    int rc = replay(d, kCallRk4Host, f_host_in, f_host_out, (const void *)(uintptr_t)dtk, nullptr, st,
                    [&](cudaStream_t s) -> int {
                      PB_CUDA(cudaMemcpyAsync(d->fstage, f_host_in, bytes, cudaMemcpyHostToDevice, s));
                      int r = stage_input(d, d->fstage, s);
                      if (r || (r = rk4_launches(d, d->fstage, dt, s))) return r;
                      PB_CUDA(cudaMemcpyAsync(f_host_out, d->fstage, bytes, cudaMemcpyDeviceToHost, s));
                      return PB_OK;
                    });
    if (rc) return rc;
    PB_CUDA(cudaStreamSynchronize(st));
    return PB_OK;
  }
  PB_CUDA(cudaMemcpyAsync(d->fstage, f_host_in, bytes, cudaMemcpyHostToDevice, st));
  int rc = pb_rtbte_rk4_step(d, d->fstage, dt, nsteps, stream);
  if (rc) return rc;
  PB_CUDA(cudaMemcpyAsync(f_host_out, d->fstage, bytes, cudaMemcpyDeviceToHost, st));
  PB_CUDA(cudaStreamSynchronize(st));
  return PB_OK;
}

extern "C" int pb_transport_setup(pb_dev *d, const double *f0, void *stream) {
  clear_error();
  if (!d || !f0) return set_error(PB_EINVAL, "pb_transport_setup: null argument");
  return ensure_weights(d, f0, (cudaStream_t)stream);
}

extern "C" int pb_transport_iterate(pb_dev *d, const double *vel3, const double *F3in, double *F3out,
                                    double *resid3, void *stream) {
  clear_error();
  if (!d || !vel3 || !F3in || !F3out) return set_error(PB_EINVAL, "pb_transport_iterate: null argument");
  if (!d->transport) return set_error(PB_EINVAL, "transport buffers were not reserved (pb_dev_opts.transport = 0)");
  cudaStream_t st = (cudaStream_t)stream;
  return replay(d, kCallTransport, vel3, F3in, F3out, resid3, st,
                [&](cudaStream_t s) { return transport_seq(d, vel3, F3in, F3out, resid3, s); });
}

extern "C" int pb_transport_iterate_host(pb_dev *d, const double *vel3, const double *F3in_host, double *F3out_host,
                                         double *resid3_host, void *stream) {
  clear_error();
  if (!d || !vel3 || !F3in_host || !F3out_host) return set_error(PB_EINVAL, "pb_transport_iterate_host: null argument");
  if (!d->transport) return set_error(PB_EINVAL, "transport buffers were not reserved (pb_dev_opts.transport = 0)");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * 3 * (size_t)d->ns;
  if (pinned_host(F3in_host) && pinned_host(F3out_host) && (!resid3_host || pinned_host(resid3_host))) {
    // page-locked buffers: the copies and the pass in one graph, replayed per buffer set
    int rc = replay(d, kCallTransportHost, vel3, F3in_host, F3out_host, resid3_host, st, [&](cudaStream_t s) -> int {
      PB_CUDA(cudaMemcpyAsync(d->Fa, F3in_host, bytes, cudaMemcpyHostToDevice, s));
      const int r = transport_seq(d, vel3, d->Fa, d->Fb, nullptr, s);
      if (r) return r;
      PB_CUDA(cudaMemcpyAsync(F3out_host, d->Fb, bytes, cudaMemcpyDeviceToHost, s));
      if (resid3_host) PB_CUDA(cudaMemcpyAsync(resid3_host, d->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
      return PB_OK;
    });
    if (rc) return rc;
    PB_CUDA(cudaStreamSynchronize(st));
    return PB_OK;
  }
  PB_CUDA(cudaMemcpyAsync(d->Fa, F3in_host, bytes, cudaMemcpyHostToDevice, st));
  // the pass Fa -> Fb, residual into the handle's scalars
  int rc = replay(d, kCallTransport, vel3, d->Fa, d->Fb, nullptr, st,
                  [&](cudaStream_t s) { return transport_seq(d, vel3, d->Fa, d->Fb, nullptr, s); });
  if (rc) return rc;
  PB_CUDA(cudaMemcpyAsync(F3out_host, d->Fb, bytes, cudaMemcpyDeviceToHost, st));
  if (resid3_host) PB_CUDA(cudaMemcpyAsync(resid3_host, d->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  PB_CUDA(cudaStreamSynchronize(st));
  return PB_OK;
}

extern "C" int pb_transport_map(pb_dev *d, const double *f0, const double *vel3, const double *F3in, double *F3out,
                                void *stream) {
  clear_error();
  if (!d || !f0 || !vel3 || !F3in || !F3out) return set_error(PB_EINVAL, "pb_transport_map: null argument");
  int rc = pb_transport_setup(d, f0, stream);
  if (rc) return rc;
  return pb_transport_iterate(d, vel3, F3in, F3out, nullptr, stream);
}

extern "C" int pb_iter_transport(pb_dev *d, const double *f0, const double *vel3, double tol, int32_t maxit,
                                 double *F3, int32_t *iters, double *resid, void *stream) {
  clear_error();
  if (!d || !f0 || !vel3 || !F3) return set_error(PB_EINVAL, "pb_iter_transport: null argument");
  if (maxit < 0 || !(tol >= 0.0)) return set_error(PB_EINVAL, "pb_iter_transport: bad tol or maxit");
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if ((rc = ensure_weights(d, f0, st))) return rc;
  const int g3 = (int)((3 * d->ns + 255) / 256);
  dev::k_tr_init<<<g3, 256, 0, st>>>(d->tau, vel3, (int)d->ns, d->Fa, d->Fff);
  PB_LAUNCHED("k_tr_init");
  if (!d->hres) {
    PB_CUDA(cudaMallocHost((void **)&d->hres, 6 * sizeof(double)));
    for (cudaEvent_t &e : d->hres_ev) PB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  double *Fbuf[2] = {d->Fa, d->Fb};  // pass i reads Fbuf[i % 2] and writes Fbuf[(i + 1) % 2]
  // pass i: replayed from one of two graphs (Fa -> Fb, Fb -> Fa), its residual numbers copied
  // to hres[3 (i % 2)] and an event recorded after them
  auto enqueue = [&](int32_t i) -> int {
    const double *Fc = Fbuf[i & 1];
    double *Fn = Fbuf[(i + 1) & 1];
    const int r = replay(d, kCallSolvePass, vel3, Fc, Fn, nullptr, st,
                         [&](cudaStream_t s) -> int { return transport_pass(d, d->Fff, vel3, Fc, Fn, d->Fff, s); });
    if (r) return r;
    PB_CUDA(cudaMemcpyAsync(d->hres + 3 * (i & 1), d->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaEventRecord(d->hres_ev[i & 1], st));
    return PB_OK;
  };
  // one pass ahead: pass i + 1 is queued before pass i's residual is read.  The extra pass after
  // the converged one only writes the other buffer (and the scratch), not the result.
  double res = INFINITY;
  int32_t it = 0;
  if (maxit > 0 && (rc = enqueue(0))) return rc;
  while (it < maxit) {
    if (it + 1 < maxit && (rc = enqueue(it + 1))) return rc;
    PB_CUDA(cudaEventSynchronize(d->hres_ev[it & 1]));
    res = d->hres[3 * (it & 1)];
    ++it;
    if (!std::isfinite(res)) break;
    if (res <= tol) break;
  }
  double *Fcur = Fbuf[it & 1];  // the iterate after `it` passes
  PB_CUDA(cudaMemcpyAsync(F3, Fcur, sizeof(double) * 3 * d->ns, cudaMemcpyDeviceToDevice, st));
  PB_CUDA(cudaStreamSynchronize(st));
  if (iters) *iters = it;
  if (resid) *resid = res;
  if (!(res <= tol))
    return set_error(PB_ENOCONV, "pb_iter_transport: relative change %.3e after %d iterations (tol %.3e)", res, it, tol);
  return PB_OK;
}

extern "C" int pb_observables(pb_dev *d, const double *f, double *out3, void *stream) {
  clear_error();
  if (!d || !f || !out3) return set_error(PB_EINVAL, "pb_observables: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = pb_collision(d, f, d->acc, stream);
  if (rc) return rc;
  dev::k_observables<<<1, 1024, 0, st>>>(f, d->eps, d->acc, (int)d->ns, out3);
  PB_LAUNCHED("k_observables");
  return PB_OK;
}

// ---------------------------------------------------------------- adjoint

namespace {

int coef_setup(pb_dev *d, cudaStream_t st) {
  if (d->variant == PB_VARIANT_FF || d->variant == PB_VARIANT_F64) {
    // per-channel coefficients and R_s on the channel plan, then (branch-merged) the sums
    // over the branches of every state pair
    const int grid = d->chan_grid(8);
    const dev::ChanGeom g = d->geom();
    const bool ff = d->variant == PB_VARIANT_FF;
    // branch-merged: the per-channel arrays hold the coefficients without g2 (the branch
    // sums multiply it back in; the |g|^2 gradient reads them as they are)
    const bool kf = d->merged;
    if (ff && kf)  dev::k_coef<true, true><<<grid, dev::kBlock, 0, st>>>(d->citems, (int)d->ncitems, g, d->ccoefA, d->ccoefB, d->cpart);
    else if (ff)   dev::k_coef<true><<<grid, dev::kBlock, 0, st>>>(d->citems, (int)d->ncitems, g, d->ccoefA, d->ccoefB, d->cpart);
    else if (kf)   dev::k_coef<false, true><<<grid, dev::kBlock, 0, st>>>(d->citems, (int)d->ncitems, g, d->ccoefA, d->ccoefB, d->cpart);
    else           dev::k_coef<false><<<grid, dev::kBlock, 0, st>>>(d->citems, (int)d->ncitems, g, d->ccoefA, d->ccoefB, d->cpart);
    PB_LAUNCHED("k_coef");
    dev::k_rowsum<<<(int)((d->ns + 255) / 256), 256, 0, st>>>(d->citem_ptr, d->cpart, (int)d->ns, d->R);
    PB_LAUNCHED("k_rowsum");
    if (d->merged && d->nsw > 0) {
      const int pg = (int)std::min<int64_t>((d->nsw + 255) / 256, 8192);
      const long long* cs = (const long long *)d->pcstart;
      if (ff) dev::k_pair_coef<true><<<pg, 256, 0, st>>>(cs, d->pcnt, (long long)d->nsw, d->ccoefA, d->ccoefB, d->coefA, d->coefB, 1.0, d->g2);
      else    dev::k_pair_coef<false><<<pg, 256, 0, st>>>(cs, d->pcnt, (long long)d->nsw, d->ccoefA, d->ccoefB, d->coefA, d->coefB, 1.0, d->g2);
      PB_LAUNCHED("k_pair_coef");
    }
    if (d->sym && !d->complete) {
      // rows that miss some partners: the tiles zeroed, then every stored pair scattered in
      const size_t tb = (size_t)d->td.nt * dev::kTile * dev::kTile * (d->c32 ? sizeof(float2) : sizeof(float4));
      void *tc = d->c32 ? (void *)d->tc32 : (void *)d->tcoef;
      PB_CUDA(cudaMemsetAsync(tc, 0, tb, st));
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((d->ns * 32 + 255) / 256, (int64_t)d->sm_count * 8));
      const long long *srp = (const long long *)d->srp;
      const float2 *cA = (const float2 *)d->coefA, *cB = (const float2 *)d->coefB;
      const int ns = (int)d->ns, nb = d->td.nb;
      if (d->c32 && d->sidx16)
        dev::k_tiles_scatter<true, uint16_t><<<grid, 256, 0, st>>>(srp, ns, d->sidx16, cA, cB, nullptr, nullptr, nb, tc);
      else if (d->c32)
        dev::k_tiles_scatter<true, uint32_t><<<grid, 256, 0, st>>>(srp, ns, d->sidx32, cA, cB, nullptr, nullptr, nb, tc);
      else if (d->sidx16)
        dev::k_tiles_scatter<false, uint16_t><<<grid, 256, 0, st>>>(srp, ns, d->sidx16, cA, cB, nullptr, nullptr, nb, tc);
      else
        dev::k_tiles_scatter<false, uint32_t><<<grid, 256, 0, st>>>(srp, ns, d->sidx32, cA, cB, nullptr, nullptr, nb, tc);
      PB_LAUNCHED("k_tiles_scatter");
    } else if (d->sym) {
      const long long n = (long long)d->td.nt * dev::kTile * dev::kTile;
      const int grid = (int)std::min<long long>((n + 255) / 256, 8192);
      if (d->c32)
        dev::k_tiles_fill_c32<<<grid, 256, 0, st>>>(d->tiles, d->td.nt, (const float2 *)d->coefA,
                                                    (const float2 *)d->coefB, (const long long *)d->srp, (int)d->ns,
                                                    d->tc32);
      else
        dev::k_tiles_fill<<<grid, 256, 0, st>>>(d->tiles, d->td.nt, (const float2 *)d->coefA,
                                                (const float2 *)d->coefB, (const long long *)d->srp, (int)d->ns,
                                                d->tcoef);
      PB_LAUNCHED("k_tiles_fill");
    }
  }
  if (d->mixed()) {
    const long long n = (long long)d->nchp;
    const int cg = (int)std::min<long long>((n + 255) / 256, 8192);
    with_g2t(d->variant, [&](auto tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      dev::k_cvt_g2<T><<<cg, 256, 0, st>>>(d->g2, n, (T *)d->g2lo, d->g2s, d->err);
    });
    PB_LAUNCHED("k_cvt_g2");
    if (d->gdense) {
      PB_CUDA(cudaMemsetAsync(d->g2d, 0, d->gd_bytes, st));
      const long long *rp = (const long long *)d->rp, *rr = (const long long *)d->rp_real;
      with_g2t(d->variant, [&](auto tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        dev::k_dense_g2<T><<<d->chan_grid(8), dev::kBlock, 0, st>>>(d->items, (int)d->nitems, rp, rr, d->col, d->g2,
                                                                    d->nmodes, d->gd_npp, (T *)d->g2d, d->g2s);
      });
      PB_LAUNCHED("k_dense_g2");
    }
  }
  return PB_OK;
}

// Mixed-precision adjoint: FP32 per-channel terms, FP64 partials and output.
int vjp_launch_mixed(pb_dev *d, const double *f, const double *lam, double wl, const double *mprev, double wm,
                     double *mu, const double *acc_in, double *acc_out, int slot, cudaStream_t st) {
  const int ns = (int)d->ns, n = (int)d->nitems;
  if (!d->vjp_g_ok)
    return set_error(PB_EINVAL, "pb_collision_vjp: the FP32/BF16/FP16 adjoint stages 20 bytes per state in shared "
                                "memory; %d states exceed it", ns);
  int rc = stage_input(d, f, st);
  if (rc) return rc;
  float *lam32 = (float *)d->vjpG;  // ns floats fit in the [ns][3] float2 table
  dev::k_vjp_prep32<<<(ns + 255) / 256, 256, 0, st>>>(f, lam, wl, mprev, wm, ns, lam32, -d->c * d->gnorm(),
                                                      slot >= 0 ? d->g2tab + (size_t)slot * ns : nullptr);
  PB_LAUNCHED("k_vjp_prep32");
  const dev::GGeom g = d->ggeom();
  const size_t smem = (sizeof(uint4) + sizeof(float)) * (size_t)ns;
  const int ctas = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(228 * 1024) / (smem + 1024)));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((d->nitems * 32 + 511) / 512, (int64_t)d->sm_count * ctas));
  if (d->gdense) {
    // the dense pair-major sweep with the rate summands weighted by lam_s - lam_p
    const int gdg = (int)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)d->gd_nitems * 32 + dev::kDenseThreads - 1) / dev::kDenseThreads, d->sm_count));
    with_g2t(d->variant, [&](auto tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      dev::k_stream_g_dense<dev::MODE_VJP, T><<<gdg, dev::kDenseThreads, smem, st>>>(
          d->gd_items, d->gd_nitems, g, (const T *)d->g2d, d->gd_npp, d->nmodes, d->gstate, ns, d->part, lam32);
    });
    PB_LAUNCHED("k_stream_g_dense (vjp)");
  } else {
    with_g2t(d->variant, [&](auto tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      dev::k_stream_g_vjp<T><<<grid, 512, smem, st>>>(d->items, n, g, (const T *)d->g2lo, d->gstate, lam32, ns, d->part);
    });
    PB_LAUNCHED("k_stream_g_vjp");
  }
  dev::k_fin_rate<true><<<fin_grid(d), kFinBlock, 0, st>>>(dev::ItemSrc{d->fwd_item_ptr(), d->part}, ns, -d->gscale(), d->R, mu);
  PB_LAUNCHED("k_fin_rate (vjp)");
  if (acc_out) {
    dev::k_lincomb<<<(ns + 255) / 256, 256, 0, st>>>(ns, 1.0, acc_in, 1.0, mu, acc_out);
    PB_LAUNCHED("k_lincomb");
  }
  return PB_OK;
}

// FF adjoint in three launches per call: vjp_prep_ff (the cotangent g = wl lam + wm mprev,
// mprev may be null, and its gather table; slot >= 0 also writes that stage of the
// |g|^2-gradient table), vjp_sweep_ff (k_stream_vjp) and vjp_fin_ff (mu = J(f)^T g, out = mu
// if not null, acc_out = acc_in + mu if not null, and the next stage's prep if nx.f is set).
int vjp_prep_ff(pb_dev *d, const double *f, const double *lam, double wl, const double *mprev, double wm,
                 double *gbuf, int slot, cudaStream_t st) {
  const int ns = (int)d->ns;
  dev::k_vjp_prep<<<(ns + 255) / 256, 256, 0, st>>>(f, lam, wl, mprev, wm, ns, gbuf, d->vjpG, -d->c,
                                                    slot >= 0 ? d->g2tab + 2 * (size_t)slot * ns : nullptr);
  PB_LAUNCHED("k_vjp_prep");
  return PB_OK;
}

int vjp_sweep_ff(pb_dev *d, cudaStream_t st) {
  const int ns = (int)d->ns, n = (int)d->nitems;
  const int grid = d->stream_grid(d->smem_G ? std::max(1, std::min(d->ctas, (int)((228 * 1024) / (d->smem_G + 1024)))) : d->ctas);
  const float4 *A4 = (const float4 *)d->coefA, *B4 = (const float4 *)d->coefB;
  if (d->smem_G) {
    if (d->sidx16) dev::k_stream_vjp<true, uint16_t><<<grid, dev::kBlock, d->smem_G, st>>>(d->items, n, A4, B4, d->sidx16, d->vjpG, ns, d->part);
    else           dev::k_stream_vjp<true, uint32_t><<<grid, dev::kBlock, d->smem_G, st>>>(d->items, n, A4, B4, d->sidx32, d->vjpG, ns, d->part);
  } else {
    if (d->sidx16) dev::k_stream_vjp<false, uint16_t><<<grid, dev::kBlock, 0, st>>>(d->items, n, A4, B4, d->sidx16, d->vjpG, ns, d->part);
    else           dev::k_stream_vjp<false, uint32_t><<<grid, dev::kBlock, 0, st>>>(d->items, n, A4, B4, d->sidx32, d->vjpG, ns, d->part);
  }
  PB_LAUNCHED("k_stream_vjp");
  return PB_OK;
}

int vjp_fin_ff(pb_dev *d, const double *gbuf, double *mu, const double *acc_in, double *acc_out,
                const dev::VjpNext &nx, cudaStream_t st) {
  const int ns = (int)d->ns;
  if (ns <= 2048)  // few states: more, smaller CTAs
    dev::k_fin_vjp<8><<<(ns + 7) / 8, 256, 0, st>>>(d->item_ptr, d->part, ns, d->c, d->R, gbuf, mu, acc_in, acc_out, nx,
                                                   d->vjpG, -d->c);
  else
    dev::k_fin_vjp<32><<<(ns + 31) / 32, 256, 0, st>>>(d->item_ptr, d->part, ns, d->c, d->R, gbuf, mu, acc_in, acc_out,
                                                      nx, d->vjpG, -d->c);
  PB_LAUNCHED("k_fin_vjp");
  return PB_OK;
}

// grad_g2 (unpadded CSR order) += dL/dg2 of the NST calls whose stages fill the table
template <int NST>
int g2grad_launch(pb_dev *d, double *grad_g2, cudaStream_t st) {
  const int ns = (int)d->ns;
  const long long *rp = (const long long *)d->rp, *rr = (const long long *)d->rp_real;
  if (d->mixed()) {
    dev::k_g2grad_g<NST><<<d->stream_grid(8), dev::kBlock, 0, st>>>(d->items, (int)d->nitems, d->ggeom(), d->gstate,
                                                                    rp, rr, d->g2tab, ns, grad_g2);
    PB_LAUNCHED("k_g2grad_g");
    return PB_OK;
  }
  const float2 *A = (const float2 *)d->ccoefA, *B = (const float2 *)d->ccoefB;
  if (d->merged) {
    // per state pair (the channel coefficients are stored without g2), on a persistent grid
    const int n = d->ngitems;
    const int gg = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)d->sm_count * dev::kGradCtas));
    const long long *pcs = (const long long *)d->pcstart;
    if (d->sidx16) dev::k_g2grad_pairs<NST, uint16_t><<<gg, dev::kBlock, 0, st>>>(d->gitems, n, d->sidx16, pcs, d->pcnt, rp, rr, A, B, d->g2tab, ns, grad_g2, d->gacc);
    else           dev::k_g2grad_pairs<NST, uint32_t><<<gg, dev::kBlock, 0, st>>>(d->gitems, n, d->sidx32, pcs, d->pcnt, rp, rr, A, B, d->g2tab, ns, grad_g2, d->gacc);
    PB_LAUNCHED("k_g2grad_pairs");
    return PB_OK;
  }
  const int gg = d->chan_grid(8), nc = (int)d->ncitems;
  if (d->col16) dev::k_g2grad<NST, uint16_t><<<gg, dev::kBlock, 0, st>>>(d->citems, nc, rp, rr, A, B, d->col16, d->g2, d->g2tab, ns, grad_g2);
  else          dev::k_g2grad<NST, uint32_t><<<gg, dev::kBlock, 0, st>>>(d->citems, nc, rp, rr, A, B, d->col, d->g2, d->g2tab, ns, grad_g2);
  PB_LAUNCHED("k_g2grad");
  return PB_OK;
}

// the deferred form: the NST stages' pair sums into the accumulators (branch-merged FF devices)
template <int NST>
int g2acc_launch(pb_dev *d, cudaStream_t st) {
  const int n = d->ngitems, ns = (int)d->ns;
  const int gg = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)d->sm_count * 8));
  if (d->sidx16) dev::k_g2acc_pairs<NST, uint16_t><<<gg, dev::kBlock, 0, st>>>(d->gitems, n, d->sidx16, d->pcnt, d->g2tab, ns, d->gacc);
  else           dev::k_g2acc_pairs<NST, uint32_t><<<gg, dev::kBlock, 0, st>>>(d->gitems, n, d->sidx32, d->pcnt, d->g2tab, ns, d->gacc);
  PB_LAUNCHED("k_g2acc_pairs");
  return PB_OK;
}

// grad_g2 += the accumulated pair sums applied to the pairs' channels (accumulators cleared)
int g2flush_launch(pb_dev *d, double *grad_g2, cudaStream_t st) {
  if (d->gaccg) {
    const long long *rp = (const long long *)d->rp, *rr = (const long long *)d->rp_real;
    dev::k_g2grad_g<0><<<d->stream_grid(8), dev::kBlock, 0, st>>>(d->items, (int)d->nitems, d->ggeom(), d->gstate,
                                                                   rp, rr, d->g2tab, (int)d->ns, grad_g2, d->gaccg);
    PB_LAUNCHED("k_g2grad_g");
    const cudaError_t e = cudaMemsetAsync(d->gaccg, 0, d->gaccg_bytes(), st);
    return e == cudaSuccess ? PB_OK : cuda_fail(e, "clear the gradient accumulators");
  }
  const int n = d->ngitems, ns = (int)d->ns;
  const int gg = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)d->sm_count * dev::kGradCtas));
  const long long *rp = (const long long *)d->rp, *rr = (const long long *)d->rp_real, *pcs = (const long long *)d->pcstart;
  const float2 *A = (const float2 *)d->ccoefA, *B = (const float2 *)d->ccoefB;
  if (d->sidx16) dev::k_g2grad_pairs<0, uint16_t><<<gg, dev::kBlock, 0, st>>>(d->gitems, n, d->sidx16, pcs, d->pcnt, rp, rr, A, B, d->g2tab, ns, grad_g2, d->gacc);
  else           dev::k_g2grad_pairs<0, uint32_t><<<gg, dev::kBlock, 0, st>>>(d->gitems, n, d->sidx32, pcs, d->pcnt, rp, rr, A, B, d->g2tab, ns, grad_g2, d->gacc);
  PB_LAUNCHED("k_g2grad_pairs");
  return PB_OK;
}

// the mixed deferred form: the NST stages' W, U, V of every (state, partner) pair
template <int NST>
int g2accg_launch(pb_dev *d, cudaStream_t st) {
  const int ns = (int)d->ns;
  if (ns == 0) return PB_OK;
  const dim3 grid((unsigned)((ns + dev::kBlock - 1) / dev::kBlock), (unsigned)std::min(ns, 65535));
  dev::k_g2acc_g<NST><<<grid, dev::kBlock, 0, st>>>(d->g2tab, ns, d->gaccg);
  PB_LAUNCHED("k_g2acc_g");
  return PB_OK;
}

int lincomb(pb_dev *d, double a, const double *x, double b, const double *y, double *out, cudaStream_t st) {
  dev::k_lincomb<<<(int)((d->ns + 255) / 256), 256, 0, st>>>((int)d->ns, a, x, b, y, out);
  PB_LAUNCHED("k_lincomb");
  return PB_OK;
}

}  // namespace

extern "C" int pb_collision_vjp(pb_dev *d, const double *f, const double *lam, double *grad_f, double *grad_g2,
                                void *stream) {
  clear_error();
  if (!d || !f || !lam || !grad_f) return set_error(PB_EINVAL, "pb_collision_vjp: null argument");
  if ((d->variant != PB_VARIANT_FF && !d->mixed()) || d->c32)
    return set_error(PB_EINVAL, "pb_collision_vjp: needs the FF, G32, G16 or H16 variant");
  cudaStream_t st = (cudaStream_t)stream;
  const int slot = grad_g2 ? 0 : -1;
  if (d->mixed()) {
    const int rc = vjp_launch_mixed(d, f, lam, 1.0, nullptr, 0.0, grad_f, nullptr, nullptr, slot, st);
    if (rc || !grad_g2) return rc;
  } else {
    int rc;
    if ((rc = vjp_prep_ff(d, f, lam, 1.0, nullptr, 0.0, d->vecs, slot, st))) return rc;
    if ((rc = vjp_sweep_ff(d, st))) return rc;
    if ((rc = vjp_fin_ff(d, d->vecs, grad_f, nullptr, nullptr, dev::VjpNext{}, st))) return rc;
    if (!grad_g2) return PB_OK;
  }
  return g2grad_launch<1>(d, grad_g2, st);
}

namespace {
// one RK4 adjoint step; defer: the |g|^2 gradient goes to the pair accumulators (FF merged)
int rk4_vjp_seq(pb_dev *d, const double *f, double *lam, double dt, double *grad_g2, bool defer, cudaStream_t st) {
  const bool want_g2 = grad_g2 || defer;
  const int64_t ns = d->ns;
  double *u2 = d->vecs, *u3 = u2 + ns, *u4 = u3 + ns, *acc = u4 + ns, *ga = acc + ns, *gb = ga + ns, *mu0 = gb + ns,
         *mu1 = mu0 + ns;
  int rc;
  // forward stages u2, u3, u4 (u1 = f) through the RK4 stage finalisers
  if ((rc = stage_input(d, f, st))) return rc;
  double *fw = const_cast<double *>(f);  // stages 0..2 only read f
  if ((rc = launch_stream(d, dev::MODE_COLL, f, d->yff, st))) return rc;
  launch_fin<0>(d, f, nullptr, fw, dt, st, u2);
  if ((rc = launch_stream(d, dev::MODE_COLL, u2, d->yff, st))) return rc;
  launch_fin<1>(d, u2, nullptr, fw, dt, st, u3);
  if ((rc = launch_stream(d, dev::MODE_COLL, u3, d->yff, st))) return rc;
  launch_fin<2>(d, u3, nullptr, fw, dt, st, u4);
  PB_LAUNCHED("rk4 vjp forward stages");
  // reverse: dL/dk4 = dt/6 lam; dL/dk3 = dt/3 lam + dt mu4; dL/dk2 = dt/3 lam + dt/2 mu3;
  // dL/dk1 = dt/6 lam + dt/2 mu2; dL/df = lam + mu1 + mu2 + mu3 + mu4, mu_i = J(u_i)^T dL/dk_i
  const double *U[4] = {f, u2, u3, u4};
  const double wl[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
  const double wm[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  if (d->mixed()) {
    double *mu = mu0, *mprev = mu1;
    for (int j = 3; j >= 0; --j) {
      std::swap(mu, mprev);
      const double *ain = j == 3 ? lam : acc;
      double *aout = j == 0 ? lam : acc;  // the last stage writes dL/df over lam (lam is read first)
      if ((rc = vjp_launch_mixed(d, U[j], lam, wl[j], j == 3 ? nullptr : mprev, wm[j], mu, ain, aout,
                                 want_g2 ? j : -1, st)))
        return rc;
    }
  } else {
    // each stage's finaliser prepares the next stage's cotangent (g alternates ga, gb)
    double *gc = ga, *gn = gb;
    if ((rc = vjp_prep_ff(d, U[3], lam, wl[3], nullptr, 0.0, gc, want_g2 ? 3 : -1, st))) return rc;
    for (int j = 3; j >= 0; --j) {
      if ((rc = vjp_sweep_ff(d, st))) return rc;
      dev::VjpNext nx{};
      if (j > 0) nx = dev::VjpNext{U[j - 1], lam, wl[j - 1], wm[j - 1], gn,
                                   want_g2 ? d->g2tab + 2 * (size_t)(j - 1) * ns : nullptr};
      // the last stage writes dL/df = lam + sum mu over lam (every read of lam precedes it)
      if ((rc = vjp_fin_ff(d, gc, nullptr, j == 3 ? lam : acc, j == 0 ? lam : acc, nx, st))) return rc;
      std::swap(gc, gn);
    }
  }
  if (defer) return d->mixed() ? g2accg_launch<4>(d, st) : g2acc_launch<4>(d, st);
  if (grad_g2 && (rc = g2grad_launch<4>(d, grad_g2, st))) return rc;
  return PB_OK;
}

// The step's launches (about 17) replayed from a graph per (lam, dt, grad_g2); f, which a
// backward pass changes from step to step, is first copied into the handle's ninth vector.
int rk4_vjp_impl(pb_dev *d, const double *f, double *lam, double dt, double *grad_g2, bool defer, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  double *fc = d->vecs + 8 * d->ns;
  PB_CUDA(cudaMemcpyAsync(fc, f, sizeof(double) * (size_t)d->ns, cudaMemcpyDeviceToDevice, st));
  uint64_t dtk = 0;
  std::memcpy(&dtk, &dt, sizeof dtk);
  return replay(d, defer ? kCallVjpDefer : kCallVjp, lam, (const void *)(uintptr_t)dtk, grad_g2, nullptr, st,
                [&](cudaStream_t s) -> int { return rk4_vjp_seq(d, fc, lam, dt, grad_g2, defer, s); });
}

int rk4_vjp_check(pb_dev *d, const double *f, const double *lam, double dt, const char *who) {
  if (!d || !f || !lam) return set_error(PB_EINVAL, "%s: null argument", who);
  if ((d->variant != PB_VARIANT_FF && !d->mixed()) || d->c32)
    return set_error(PB_EINVAL, "%s: needs the FF, G32, G16 or H16 variant", who);
  if (!std::isfinite(dt)) return set_error(PB_EINVAL, "%s: bad dt", who);
  return PB_OK;
}
}  // namespace

extern "C" int pb_rtbte_rk4_vjp(pb_dev *d, const double *f, double *lam, double dt, double *grad_g2, void *stream) {
  clear_error();
  if (int rc = rk4_vjp_check(d, f, lam, dt, "pb_rtbte_rk4_vjp")) return rc;
  return rk4_vjp_impl(d, f, lam, dt, grad_g2, false, stream);
}

extern "C" int pb_rtbte_rk4_vjp_defer(pb_dev *d, const double *f, double *lam, double dt, void *stream) {
  clear_error();
  if (int rc = rk4_vjp_check(d, f, lam, dt, "pb_rtbte_rk4_vjp_defer")) return rc;
  if (!d->gacc && !d->gaccg)
    return set_error(PB_EINVAL, "pb_rtbte_rk4_vjp_defer: needs a device created with adjoint = 1 (FF branch-merged, G32, G16 or H16)");
  return rk4_vjp_impl(d, f, lam, dt, nullptr, true, stream);
}

extern "C" int pb_dev_g2grad_flush(pb_dev *d, double *grad_g2, void *stream) {
  clear_error();
  if (!d || !grad_g2) return set_error(PB_EINVAL, "pb_dev_g2grad_flush: null argument");
  if (!d->gacc && !d->gaccg) return set_error(PB_EINVAL, "pb_dev_g2grad_flush: the device keeps no gradient accumulators");
  return g2flush_launch(d, grad_g2, (cudaStream_t)stream);
}

extern "C" int pb_dev_set_g2(pb_dev *d, const double *g2, void *stream) {
  clear_error();
  if (!d || !g2) return set_error(PB_EINVAL, "pb_dev_set_g2: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  dev::k_set_g2<<<d->chan_grid(8), dev::kBlock, 0, st>>>(d->citems, (int)d->ncitems, (const long long *)d->rp,
                                                           (const long long *)d->rp_real, g2, d->g2);
  PB_LAUNCHED("k_set_g2");
  if (d->sym) {
    // the caller may give the two stored copies of a channel different values: the symmetric
    // tiles (which take a pair's reverse from its own entry) no longer apply; stream rows
    d->sym = false;
    drop_rk_graphs(d);
  }
  d->drop_call_graphs();  // the calls' launch sequences are captured again on their next use
  return coef_setup(d, st);
}

// ---------------------------------------------------------------- no-allocation collision
//
// pb_collision_static: the collision sweep for callers that may not allocate device
// memory.  Its per-call scratch (the float-float copy of f and one partial per work
// item) lives in this file-scope device array instead of the arena's scratch regions.
// Every GPU that loads the library holds the array until the process exits.  In host
// code the symbol only names the array; its device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
static __device__ __align__(256) unsigned char pb_static_scratch[PB_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
// per device: the context the address was looked up in (its process-unique id) and the address
struct StaticAddr {
  unsigned long long ctx = 0;
  void *addr = nullptr;
};
StaticAddr g_static_addr[kMaxStaticDevices];

// The unique id of the calling thread's current context (cuCtxGetCurrent + cuCtxGetId, reached
// through the runtime's driver entry points so that the library does not link the driver
// library); 0 when there is none or the lookup is unavailable.  A device reset or a new primary
// context gets a new id, and with it a new lookup of the array's address.
typedef CUresult(CUDAAPI *CtxGetCurrentFn)(CUcontext *);
typedef CUresult(CUDAAPI *CtxGetIdFn)(CUcontext, unsigned long long *);
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
    cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int static_scratch_address(void **out) {
  int devid = 0;
  PB_CUDA(cudaGetDevice(&devid));
  if (devid < 0 || devid >= kMaxStaticDevices)
    return set_error(PB_EDEVICE, "pb_collision_static: device %d is beyond the %d devices it tracks", devid,
                     kMaxStaticDevices);
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticAddr &a = g_static_addr[devid];
  const unsigned long long ctx = current_ctx_id();
  if (!a.addr || ctx == 0 || ctx != a.ctx) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, pb_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "pb_collision_static: cudaGetSymbolAddress");
    a.addr = p;
    a.ctx = current_ctx_id();  // the lookup made the device's primary context current if none was
  }
  *out = a.addr;
  return PB_OK;
}

}  // namespace

extern "C" int pb_collision_static(pb_dev *d, const double *f, double *dfdt, void *stream) {
  clear_error();
  if (!d || !f || !dfdt) return set_error(PB_EINVAL, "pb_collision_static: null argument");
  if (d->mixed() || d->variant == PB_VARIANT_PAPER)
    return set_error(PB_EINVAL, "pb_collision_static: available for the FF, F64 and literal variants only");
  const size_t ff_bytes = align_up(sizeof(float2) * (size_t)d->ns);
  const size_t part_bytes = sizeof(Part4) * (size_t)d->nitems;
  if (ff_bytes + part_bytes > (size_t)PB_STATIC_SCRATCH_BYTES)
    return set_error(PB_EINVAL,
                     "pb_collision_static: this problem needs %zu bytes of scratch (%lld states, %lld work items) "
                     "but the static array holds %zu bytes; use pb_collision or larger work items",
                     ff_bytes + part_bytes, (long long)d->ns, (long long)d->nitems, (size_t)PB_STATIC_SCRATCH_BYTES);
  void *base = nullptr;
  int rc = static_scratch_address(&base);
  if (rc) return rc;
  float2 *fff = (float2 *)base;
  Part4 *part = (Part4 *)((char *)base + ff_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  if (d->variant == PB_VARIANT_FF && (rc = to_ff(d, f, d->ns, fff, st))) return rc;
  if ((rc = launch_stream_to(d, dev::MODE_COLL, f, fff, part, st))) return rc;
  PB_LAUNCHED("pb_collision_static: stream kernel");
  if (d->variant == PB_VARIANT_LITERAL)
    dev::k_fin_coll<true, -1><<<fin_grid(d), kFinBlock, 0, st>>>(dev::ItemSrc{d->item_ptr, part}, (int)d->ns, d->c, d->R, f, dfdt,
                                                                 nullptr, nullptr, nullptr, nullptr, 0.0);
  else
    dev::k_fin_coll<false, -1><<<fin_grid(d), kFinBlock, 0, st>>>(dev::ItemSrc{d->item_ptr, part}, (int)d->ns, d->c, d->R, f, dfdt,
                                                                  nullptr, nullptr, nullptr, nullptr, 0.0);
  PB_LAUNCHED("pb_collision_static: k_fin_coll");
  return PB_OK;
}

// ---------------------------------------------------------------- batched rt-BTE
#include "batch.cuh"
