/*
 * Seeded synthetic |g|^2 generator.
 *
 * Input generation only: this file holds none of the collision-integral
 * arithmetic.  It stands in for the first-principles e-ph couplings
 * |g_{mn nu}(k,q)|^2 of the paper's Eq. 2, which are inputs there (they come
 * from DFT interpolation, outside the BTE solver).  Both the CPU oracle and the
 * GPU library receive the values it produces.
 *
 * Value:  g2 = exp(mu + sigma_ln * Z),  Z ~ N(0,1) by Box-Muller from two
 * uniforms drawn from a splitmix64 hash of a canonical channel key.
 *
 * Canonical key.  A channel joins state s = (n,k) to state p = (m,k') through
 * phonon branch nu.  The key is made invariant under
 *   - the swap s <-> p  (so |g|^2 is symmetric under k <-> k+q),
 *   - the 48 operations of the cubic point group O_h acting on k and k'
 *     together (independent sign flips of each axis, permutations of axes;
 *     the permutations only when all three grid sizes are equal).
 * Each axis contributes the pair (k_i, k'_i) taken modulo N_i; the sign flip of
 * that axis maps it to (-k_i, -k'_i) mod N_i, so the smaller of the two pairs
 * is invariant.  Sorting the three per-axis pairs removes the permutation.  The
 * invariance makes the synthetic problem cubic- and inversion-symmetric, like
 * the tight-binding bands and phonons built in synth/__init__.py.
 *
 * State ids are full-grid ids: id = ik * nbands + n with
 * ik = (j1 * N2 + j2) * N3 + j3 and k_i = 2 pi j_i / N_i.
 */
#include <math.h>
#include <stdint.h>

typedef struct {
  int32_t nk[3];
  int32_t nbands;
  int32_t nmodes;
  int32_t cubic; /* 1: also symmetrise under axis permutations (needs N1=N2=N3) */
  double mu;       /* mean of ln|g|^2, |g|^2 in eV^2 */
  double sigma_ln; /* standard deviation of ln|g|^2 */
  uint64_t seed;
} synth_g2_params;

static inline uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* per-axis pair (a, b) in [0,N)^2, canonical under simultaneous negation */
static inline uint64_t axis_pair(int32_t a, int32_t b, int32_t N) {
  int32_t na = (N - a) % N, nb = (N - b) % N;
  uint64_t x = (uint64_t)a * (uint64_t)N + (uint64_t)b;
  uint64_t y = (uint64_t)na * (uint64_t)N + (uint64_t)nb;
  return x < y ? x : y;
}

static inline void sort3(uint64_t v[3]) {
  uint64_t t;
  if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
  if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
  if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

/* key of the ordered channel (n,k) -> (m,k'): 5 words (n, m, pair1..3) */
static void ordered_key(const synth_g2_params *P, int32_t n, const int32_t j[3], int32_t m,
                        const int32_t jp[3], uint64_t out[5]) {
  uint64_t pr[3];
  for (int i = 0; i < 3; ++i) pr[i] = axis_pair(j[i], jp[i], P->nk[i]);
  if (P->cubic) sort3(pr);
  out[0] = (uint64_t)n;
  out[1] = (uint64_t)m;
  out[2] = pr[0];
  out[3] = pr[1];
  out[4] = pr[2];
}

static inline void decode(const synth_g2_params *P, int32_t id, int32_t *n, int32_t j[3]) {
  int32_t nb = P->nbands;
  *n = id % nb;
  int32_t ik = id / nb;
  j[2] = ik % P->nk[2];
  j[1] = (ik / P->nk[2]) % P->nk[1];
  j[0] = ik / (P->nk[2] * P->nk[1]);
}

double synth_g2(int32_t s, int32_t p, int32_t nu, const void *user) {
  const synth_g2_params *P = (const synth_g2_params *)user;
  int32_t n, m, j[3], jp[3];
  decode(P, s, &n, j);
  decode(P, p, &m, jp);
  uint64_t a[5], b[5];
  ordered_key(P, n, j, m, jp, a);
  ordered_key(P, m, jp, n, j, b);
  const uint64_t *k = a;
  for (int i = 0; i < 5; ++i) {
    if (a[i] != b[i]) { k = (a[i] < b[i]) ? a : b; break; }
  }
  uint64_t h = splitmix64(P->seed);
  h = splitmix64(h ^ (uint64_t)(uint32_t)nu);
  for (int i = 0; i < 5; ++i) h = splitmix64(h ^ k[i]);
  uint64_t h1 = splitmix64(h ^ 0x5555555555555555ULL);
  uint64_t h2 = splitmix64(h ^ 0xaaaaaaaaaaaaaaaaULL);
  double u1 = ((double)(h1 >> 11) + 1.0) * 0x1.0p-53; /* (0, 1] */
  double u2 = (double)(h2 >> 11) * 0x1.0p-53;         /* [0, 1) */
  double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  return exp(P->mu + P->sigma_ln * z);
}

/* batched form; matches the pb_g2_fn callback shape of the GPU library */
int synth_g2_batch(int64_t n, const int32_t *s, const int32_t *p, const int32_t *nu, double *out,
                   void *user) {
  for (int64_t i = 0; i < n; ++i) out[i] = synth_g2(s[i], p[i], nu[i], user);
  return 0;
}

/* fill an array for every (s, p, nu) of the given id lists: out[(i*np + j)*nm + nu] */
void synth_g2_dense(int32_t ns, const int32_t *s, int32_t np, const int32_t *p, int32_t nm,
                    double *out, const void *user) {
  for (int32_t i = 0; i < ns; ++i)
    for (int32_t j = 0; j < np; ++j)
      for (int32_t v = 0; v < nm; ++v) out[((int64_t)i * np + j) * nm + v] = synth_g2(s[i], p[j], v, user);
}
