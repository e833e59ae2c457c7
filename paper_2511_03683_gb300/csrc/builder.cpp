// Host channel builder: the paper's step 1 ("create the target layer", Sec.
// "Optimized GPU algorithm"), which it performs once on the CPU.  Here it selects
// the energy-window states, enumerates every scattering channel (k, q, n, m, nu)
// between two window states with a positive phonon energy (Sec. "Collision integral,
// e-ph coupling matrix, and scattering channels": commensurate k/q grids, energy
// window, |g| cutoff), asks the caller for |g|^2, and lays the channels out as a
// state-segmented CSR list in which every channel appears under both of its states.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "pb_internal.h"

namespace pb {

static thread_local std::string g_err;

int set_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

const char *last_error() { return g_err.c_str(); }

}  // namespace pb

using namespace pb;

extern "C" const char *pb_last_error(void) { return pb::last_error(); }

extern "C" const char *pb_version(void) { return "pb 0.1 sm_103a"; }

namespace {

int nthreads_of(const pb_build_opts *o) {
#ifdef _OPENMP
  if (o && o->nthreads > 0) return o->nthreads;
  return omp_get_max_threads();
#else
  (void)o;
  return 1;
#endif
}

inline int64_t q_index(const int32_t *nk, int64_t iks, int64_t ikp) {
  const int64_t N2 = nk[1], N3 = nk[2];
  const int64_t s1 = iks / (N2 * N3), s2 = (iks / N3) % N2, s3 = iks % N3;
  const int64_t p1 = ikp / (N2 * N3), p2 = (ikp / N3) % N2, p3 = ikp % N3;
  const int64_t q1 = (p1 - s1 + nk[0]) % nk[0], q2 = (p2 - s2 + N2) % N2, q3 = (p3 - s3 + N3) % N3;
  return (q1 * N2 + q2) * N3 + q3;
}

}  // namespace

extern "C" int pb_build_channels(const pb_model *m, pb_g2_fn g2fn, void *user, const pb_build_opts *opts,
                                 pb_channels **out) {
  clear_error();
  if (!m || !g2fn || !out) return set_error(PB_EINVAL, "pb_build_channels: null model, callback or output");
  *out = nullptr;
  if (m->nk[0] < 1 || m->nk[1] < 1 || m->nk[2] < 1)
    return set_error(PB_EINVAL, "pb_build_channels: grid dimensions must be >= 1");
  if (m->nbands < 1 || m->nbands > 255 || m->nmodes < 1 || m->nmodes > 255)
    return set_error(PB_EINVAL, "pb_build_channels: nbands and nmodes must be in 1..255");
  if (!m->eps || !m->omega) return set_error(PB_EINVAL, "pb_build_channels: eps and omega are required");
  if (!(m->T > 0.0) || !(m->sigma > 0.0) || !std::isfinite(m->T) || !std::isfinite(m->sigma))
    return set_error(PB_EINVAL, "pb_build_channels: T and sigma must be positive and finite");
  const double g2_min = opts ? opts->g2_min : 0.0;
  const double dlim = (opts && opts->delta_nsigma > 0.0) ? opts->delta_nsigma * m->sigma : 0.0;
  const bool check = opts ? opts->check_closure != 0 : true;
  const bool cb_parallel = opts ? opts->callback_threadsafe != 0 : false;
  const int nt = nthreads_of(opts);

  const int64_t nq = (int64_t)m->nk[0] * m->nk[1] * m->nk[2];
  const int32_t nb = m->nbands, nm = m->nmodes;
  const int64_t nfull = nq * nb;
  if (nfull > INT32_MAX) return set_error(PB_EINVAL, "pb_build_channels: grid too large for 32-bit state ids");
  for (int64_t i = 0; i < nfull; ++i)
    if (!std::isfinite(m->eps[i])) return set_error(PB_EINVAL, "pb_build_channels: non-finite eps[%lld]", (long long)i);
  for (int64_t i = 0; i < nq * nm; ++i)
    if (!std::isfinite(m->omega[i])) return set_error(PB_EINVAL, "pb_build_channels: non-finite omega[%lld]", (long long)i);

  pb_channels *ch = new (std::nothrow) pb_channels();
  if (!ch) return set_error(PB_ENOMEM, "pb_build_channels: out of host memory");
  try {
    for (int i = 0; i < 3; ++i) ch->nk[i] = m->nk[i];
    ch->nbands = nb;
    ch->nmodes = nm;
    ch->nq = nq;
    ch->T = m->T;
    ch->sigma = m->sigma;
    ch->omega.assign(m->omega, m->omega + nq * nm);

    // window states, ascending full-grid id
    std::vector<int32_t> widx((size_t)nfull, -1);
    for (int64_t id = 0; id < nfull; ++id) {
      const int32_t n = (int32_t)(id % nb);
      const double e = m->eps[id];
      const bool in = !m->win || (e >= m->win[2 * n] && e <= m->win[2 * n + 1]);
      if (in) {
        widx[id] = (int32_t)ch->state_ids.size();
        ch->state_ids.push_back((int32_t)id);
      }
    }
    const int64_t ns = (int64_t)ch->state_ids.size();
    if (ns == 0) {
      delete ch;
      return set_error(PB_EINVAL, "pb_build_channels: the energy window holds no state");
    }
    if (ns >= kMaxStates) {
      delete ch;
      return set_error(PB_EINVAL, "pb_build_channels: %lld window states exceed the 2^24 limit", (long long)ns);
    }
    ch->nstate = ns;
    ch->kidx.resize(ns);
    ch->eps.resize(ns);
    if (m->vel) ch->vel.resize(3 * ns);
    for (int64_t r = 0; r < ns; ++r) {
      const int32_t id = ch->state_ids[r];
      ch->kidx[r] = id / nb;
      ch->eps[r] = m->eps[id];
      if (m->vel)
        for (int a = 0; a < 3; ++a) ch->vel[3 * r + a] = m->vel[3 * (int64_t)id + a];
    }

    // phonon branches with positive energy, per q
    std::vector<uint8_t> npos((size_t)nq);
    for (int64_t q = 0; q < nq; ++q) {
      int c = 0;
      for (int v = 0; v < nm; ++v) c += ch->omega[q * nm + v] > 0.0;
      npos[q] = (uint8_t)c;
    }

    // approximate energy conservation (the paper's delta cutoff, optional): keep a channel
    // unless both Gaussian arguments x + w and x - w lie beyond dlim
    auto keep_delta = [&](int64_t r, int64_t p, int64_t q, int v) {
      if (dlim <= 0.0) return true;
      const double x = ch->eps[r] - ch->eps[p], w = ch->omega[q * nm + v];
      return !(std::fabs(x + w) > dlim && std::fabs(x - w) > dlim);
    };
    // row lengths, then the CSR offsets
    std::vector<int64_t> len((size_t)ns);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
    for (int64_t r = 0; r < ns; ++r) {
      int64_t c = 0;
      const int64_t iks = ch->kidx[r];
      for (int64_t p = 0; p < ns; ++p) {
        const int64_t q = q_index(m->nk, iks, ch->kidx[p]);
        if (dlim <= 0.0) {
          c += npos[q];
          continue;
        }
        for (int v = 0; v < nm; ++v)
          if (ch->omega[q * nm + v] > 0.0 && keep_delta(r, p, q, v)) ++c;
      }
      len[r] = c;
    }
    ch->row_ptr.assign(ns + 1, 0);
    for (int64_t r = 0; r < ns; ++r) ch->row_ptr[r + 1] = ch->row_ptr[r] + len[r];
    int64_t nch = ch->row_ptr[ns];
    ch->col.resize(nch);
    ch->nu.resize(nch);
    ch->g2.resize(nch);

#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
    for (int64_t r = 0; r < ns; ++r) {
      int64_t c = ch->row_ptr[r];
      const int64_t iks = ch->kidx[r];
      for (int64_t p = 0; p < ns; ++p) {
        const int64_t q = q_index(m->nk, iks, ch->kidx[p]);
        for (int v = 0; v < nm; ++v)
          if (ch->omega[q * nm + v] > 0.0 && keep_delta(r, p, q, v)) {
            ch->col[c] = (int32_t)p;
            ch->nu[c] = (uint8_t)v;
            ++c;
          }
      }
    }

    // |g|^2 from the caller, one row per callback
    int cb_status = 0;
    int64_t bad = -1;
    auto fill_row = [&](int64_t r, std::vector<int32_t> &sb, std::vector<int32_t> &pb_, std::vector<int32_t> &vb) {
      const int64_t a = ch->row_ptr[r], n = ch->row_ptr[r + 1] - a;
      if (n == 0) return 0;
      sb.assign(n, ch->state_ids[r]);
      pb_.resize(n);
      vb.resize(n);
      for (int64_t i = 0; i < n; ++i) {
        pb_[i] = ch->state_ids[ch->col[a + i]];
        vb[i] = ch->nu[a + i];
      }
      int rc = g2fn(n, sb.data(), pb_.data(), vb.data(), ch->g2.data() + a, user);
      if (rc) return 1;
      for (int64_t i = 0; i < n; ++i) {
        const double g = ch->g2[a + i];
        if (!(g >= 0.0) || !std::isfinite(g)) return 2;
      }
      return 0;
    };
    if (cb_parallel) {
#pragma omp parallel num_threads(nt)
      {
        std::vector<int32_t> sb, pb_, vb;
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < ns; ++r) {
          int rc = fill_row(r, sb, pb_, vb);
          if (rc) {
#pragma omp critical
            {
              cb_status = rc;
              bad = r;
            }
          }
        }
      }
    } else {
      std::vector<int32_t> sb, pb_, vb;
      for (int64_t r = 0; r < ns && !cb_status; ++r) {
        cb_status = fill_row(r, sb, pb_, vb);
        if (cb_status) bad = r;
      }
    }
    if (cb_status) {
      delete ch;
      return set_error(PB_ECALLBACK, cb_status == 1 ? "pb_build_channels: g2 callback failed on row %lld"
                                                    : "pb_build_channels: g2 callback gave a negative or non-finite value on row %lld",
                       (long long)bad);
    }

    // optional |g| cutoff: compact the rows
    if (g2_min > 0.0) {
      std::vector<int64_t> rp2(ns + 1, 0);
      int64_t w = 0;
      for (int64_t r = 0; r < ns; ++r) {
        for (int64_t c = ch->row_ptr[r]; c < ch->row_ptr[r + 1]; ++c)
          if (ch->g2[c] >= g2_min) {
            ch->col[w] = ch->col[c];
            ch->nu[w] = ch->nu[c];
            ch->g2[w] = ch->g2[c];
            ++w;
          }
        rp2[r + 1] = w;
      }
      ch->row_ptr.swap(rp2);
      nch = w;
      ch->col.resize(nch);
      ch->nu.resize(nch);
      ch->g2.resize(nch);
      ch->col.shrink_to_fit();
      ch->nu.shrink_to_fit();
      ch->g2.shrink_to_fit();
    }
    ch->nch = nch;
    int64_t mx = 0;
    for (int64_t r = 0; r < ns; ++r) mx = std::max(mx, ch->row_ptr[r + 1] - ch->row_ptr[r]);
    ch->max_row = mx;

    // closure: the reverse channel (p -> s, same branch) exists with the same |g|^2
    if (check) {
      int64_t fail = -1;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 8)
      for (int64_t r = 0; r < ns; ++r) {
        for (int64_t c = ch->row_ptr[r]; c < ch->row_ptr[r + 1]; ++c) {
          const int32_t p = ch->col[c];
          const uint8_t v = ch->nu[c];
          const int32_t *b = ch->col.data() + ch->row_ptr[p];
          const int32_t *e = ch->col.data() + ch->row_ptr[p + 1];
          const int32_t *lo = std::lower_bound(b, e, (int32_t)r);
          bool ok = false;
          for (const int32_t *it = lo; it != e && *it == (int32_t)r; ++it) {
            const int64_t cc = it - ch->col.data();
            if (ch->nu[cc] == v) {
              ok = ch->g2[cc] == ch->g2[c];
              break;
            }
          }
          if (!ok) {
#pragma omp critical
            fail = c;
          }
        }
      }
      if (fail >= 0) {
        delete ch;
        return set_error(PB_ENOTCLOSED, "pb_build_channels: channel %lld has no reverse channel with equal |g|^2",
                         (long long)fail);
      }
      ch->closed = true;
    }
  } catch (const std::bad_alloc &) {
    delete ch;
    return set_error(PB_ENOMEM, "pb_build_channels: out of host memory");
  }
  *out = ch;
  return PB_OK;
}

extern "C" int pb_channels_get_info(const pb_channels *ch, pb_channels_info *info) {
  clear_error();
  if (!ch || !info) return set_error(PB_EINVAL, "pb_channels_get_info: null argument");
  std::memset(info, 0, sizeof *info);
  info->nstate = ch->nstate;
  info->nchannels = ch->nch;
  info->nq = ch->nq;
  for (int i = 0; i < 3; ++i) info->nk[i] = ch->nk[i];
  info->nbands = ch->nbands;
  info->nmodes = ch->nmodes;
  info->T = ch->T;
  info->sigma = ch->sigma;
  info->max_row = ch->max_row;
  return PB_OK;
}

extern "C" int pb_channels_export(const pb_channels *ch, int64_t *row_ptr, int32_t *col, int32_t *nu, double *g2,
                                  int32_t *state_ids) {
  clear_error();
  if (!ch) return set_error(PB_EINVAL, "pb_channels_export: null handle");
  if (row_ptr) std::memcpy(row_ptr, ch->row_ptr.data(), sizeof(int64_t) * (ch->nstate + 1));
  if (col) std::memcpy(col, ch->col.data(), sizeof(int32_t) * ch->nch);
  if (nu)
    for (int64_t i = 0; i < ch->nch; ++i) nu[i] = ch->nu[i];
  if (g2) std::memcpy(g2, ch->g2.data(), sizeof(double) * ch->nch);
  if (state_ids) std::memcpy(state_ids, ch->state_ids.data(), sizeof(int32_t) * ch->nstate);
  return PB_OK;
}

extern "C" void pb_channels_free(pb_channels *ch) { delete ch; }
