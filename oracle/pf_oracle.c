/*
 * pf_oracle.c -- plain, slow FP64 CPU oracle for one RNA / ARNA
 * particle-filter time step (propagate, Gaussian-PSF likelihood, per-group
 * systematic resampling, ring exchange).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or constant generator with the CUDA library, and it includes nothing
 * from it.  The two sides agree only through the written definitions cited
 * below.
 *
 * Paper: O. Demirel, I. Smal, W. Niessen, E. Meijering, I. F. Sbalzarini,
 * "An Adaptive Distributed Resampling Algorithm with Non-Proportional
 * Allocation" (arXiv:1310.4624).  "Alg. 1" is SIR, "Alg. 2" is RNA,
 * "Alg. 3" is ARNA, "Eq. 3" is the adaptive exchange count and "Eq. 4" is
 * PE_eff.
 *
 * Precision: FP64 everywhere, except the one place where floating point
 * decides an integer that must match the GPU bit for bit: the fixed-point
 * weight code q of the resampler (ora_quantize).  That decision is taken in
 * FP32 with the fully specified operation sequence given there.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), key = (seed_lo, seed_hi), counter
 * (c0, c1, c2, c3) with c3 = track << 8 | stream << 4 | call.  Streams:
 * INIT 0, PROP 1, RESAMPLE 2, RING 3, EXCH 4.
 *
 * Parity status: every exported function is pinned by a test against a
 * closed form, an invariant, an installed library routine or brute force,
 * except the initial-population samplers (ora_init), which are pinned by
 * Kolmogorov-Smirnov tests against their laws (statistically).
 *
 * Build: plain C11, no contraction of a*b+c into fma (-ffp-contract=off) so
 * that x86-64 and AArch64 hosts give identical results.
 *
 * Threads: with OpenMP (-fopenmp) the per-particle and per-group loops of
 * ora_step can run on several host threads (ora_set_threads; 1 by default).
 * Every such loop writes only its own item's outputs and sums within an
 * item in the serial order, so the results do not depend on the thread
 * count.  This exists to time the oracle on all host cores beside the GPU.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads of ora_step's parallel loops (see "Threads" above). */
static int ora_threads = 1;

/* Set the thread count of the parallel loops (n >= 1); returns the count in
 * effect, 1 when the library was built without OpenMP. */
int ora_set_threads(int n) {
#ifdef _OPENMP
  ora_threads = n < 1 ? 1 : n;
  return ora_threads;
#else
  (void)n;
  return 1;
#endif
}

#define ORA_STREAM_INIT 0u
#define ORA_STREAM_PROP 1u
#define ORA_STREAM_RESAMPLE 2u
#define ORA_STREAM_RING 3u
#define ORA_STREAM_EXCH 4u

#define ORA_RNA 0
#define ORA_ARNA 1

#define ORA_OBS_IMAGE 0
#define ORA_OBS_POINT 1
#define ORA_OBS_FRAME 2

#define ORA_TOPO_RING 0
#define ORA_TOPO_NODE_RING 1
#define ORA_TOPO_HYPERCUBE 2

#define ORA_SEND_SYSTEMATIC 0
#define ORA_SEND_KEYED 1

#define ORA_RESAMPLE_ALWAYS 0
#define ORA_RESAMPLE_ESS 1

#define ORA_INIT_POINT 0
#define ORA_INIT_UNIFORM 1
#define ORA_INIT_SHARING 2

#define ORA_PI 3.14159265358979323846
#define ORA_LN2 0.69314718055994530942

typedef unsigned __int128 u128;

/* Filter configuration for one track, as the oracle sees it. */
typedef struct {
  int32_t G, Np, H, W;
  int32_t R;        /* patch radius: the likelihood patch is (2R+1)^2 pixels */
  int32_t mode;     /* ORA_RNA or ORA_ARNA */
  int32_t obs_kind; /* ORA_OBS_IMAGE (patch residual), ORA_OBS_FRAME (frame likelihood ratio) or ORA_OBS_POINT */
  int32_t resample_rule; /* ORA_RESAMPLE_ALWAYS (Alg. 2/3) or ORA_RESAMPLE_ESS (Alg. 1's N_eff test per group) */
  double sigma_psf, background, sigma_obs;
  double sigma_pos, sigma_v, sigma_I;
  double ex_ratio; /* RNA: fixed N_ex / N_p */
  double cutoff;   /* ARNA: no exchange once PE_eff >= cutoff * G */
  uint64_t seed;
  uint32_t track;
  int32_t send_rule;   /* ORA_SEND_SYSTEMATIC or ORA_SEND_KEYED (which slots a group sends) */
  double ess_fraction; /* ORA_RESAMPLE_ESS: N_thresh = ess_fraction * Np */
  int32_t topology;    /* ORA_TOPO_RING, ORA_TOPO_NODE_RING or ORA_TOPO_HYPERCUBE (Sec. VI) */
  int32_t node_groups; /* ORA_TOPO_NODE_RING: groups per node */
} ora_cfg;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 5): ten rounds of two 32x32->64 multiplies,   */
/* Weyl-sequence key schedule.                                              */
/* ------------------------------------------------------------------------ */
void ora_philox(uint64_t seed, const uint32_t ctr[4], uint32_t out[4]) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_stream(const ora_cfg* c, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t stream, uint32_t call, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, (c->track << 8) | (stream << 4) | call};
  ora_philox(c->seed, ctr, out);
}

/* Uniform in (0,1): the top 23 bits of a word, centred in their cell,
 * ((w >> 9) + 1/2) 2^-23.  Every value has at most 24 significant bits, so
 * the same number is exact in FP32 and FP64. */
double ora_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Bounded integer in [0, s) by Lemire's multiply-shift with rejection
 * (D. Lemire, "Fast random integer generation in an interval", ACM TOMACS
 * 2019).  Returns 1 and writes *out when the word is accepted, 0 when it is
 * rejected (the caller then draws a fresh word). */
int ora_bounded(uint32_t w, uint32_t s, uint32_t* out) {
  uint64_t m = (uint64_t)w * (uint64_t)s;
  uint32_t l = (uint32_t)m;
  if (l < s) {
    uint32_t t = (uint32_t)(0u - s) % s;
    if (l < t) return 0;
  }
  *out = (uint32_t)(m >> 32);
  return 1;
}

void ora_bounded_batch(const uint32_t* w, int64_t n, uint32_t s, int32_t* out) {
  for (int64_t i = 0; i < n; ++i) {
    uint32_t v;
    out[i] = ora_bounded(w[i], s, &v) ? (int32_t)v : -1;
  }
}

/* A uniform integer in [0, s) for (stream, call, index c0, step k): attempt
 * a uses counter (c0, a, k, tag | call) word 0; rejected attempts move on to
 * a + 1. */
static uint32_t draw_bounded_call(const ora_cfg* c, uint32_t stream, uint32_t call, uint32_t c0, uint32_t k,
                                  uint32_t s) {
  for (uint32_t a = 0;; ++a) {
    uint32_t w[4], v;
    philox_stream(c, c0, a, k, stream, call, w);
    if (ora_bounded(w[0], s, &v)) return v;
  }
}

uint32_t ora_draw_bounded(const ora_cfg* c, uint32_t stream, uint32_t c0, uint32_t k, uint32_t s) {
  return draw_bounded_call(c, stream, 0u, c0, k, s);
}

/* Five standard normals for the particle in slot j of group g at step k, by
 * Box-Muller: rho = sqrt(-2 ln u_a), (rho cos 2 pi u_b, rho sin 2 pi u_b).
 * Call 0 gives eps_x, eps_y (words 0,1) and eps_vx, eps_vy (words 2,3); call 1
 * words 0,1 give eps_I (the sine partner is not used). */
void ora_normals(const ora_cfg* c, uint32_t g, uint32_t j, uint32_t k, double eps[5]) {
  uint32_t a[4], b[4];
  philox_stream(c, j, g, k, ORA_STREAM_PROP, 0u, a);
  philox_stream(c, j, g, k, ORA_STREAM_PROP, 1u, b);
  double r0 = sqrt(-2.0 * log(ora_uniform(a[0])));
  double t0 = 2.0 * ORA_PI * ora_uniform(a[1]);
  double r1 = sqrt(-2.0 * log(ora_uniform(a[2])));
  double t1 = 2.0 * ORA_PI * ora_uniform(a[3]);
  double r2 = sqrt(-2.0 * log(ora_uniform(b[0])));
  double t2 = 2.0 * ORA_PI * ora_uniform(b[1]);
  eps[0] = r0 * cos(t0);
  eps[1] = r0 * sin(t0);
  eps[2] = r1 * cos(t1);
  eps[3] = r1 * sin(t1);
  eps[4] = r2 * cos(t2);
}

/* ------------------------------------------------------------------------ */
/* S1: ring topology (Sec. III-C; Sec. IV-B; Alg. 3 step 1).                */
/* ------------------------------------------------------------------------ */

/* Fisher-Yates on the identity, descending: for j = G-1 .. 1 swap entries j
 * and r[j], r[j] in [0, j]. */
void ora_fisher_yates(int32_t G, const uint32_t* r, int32_t* sigma) {
  for (int32_t g = 0; g < G; ++g) sigma[g] = g;
  for (int32_t j = G - 1; j >= 1; --j) {
    int32_t t = sigma[j];
    sigma[j] = sigma[r[j]];
    sigma[r[j]] = t;
  }
}

/* Hypercube dimensions: ceil(log2 G). */
int32_t ora_hyper_dims(int32_t G) {
  int32_t D = 0;
  while ((1 << D) < G) ++D;
  return D;
}

/* Communication topology of step k (Sec. IV-B; Sec. VI for the others).
 * ORA_TOPO_RING: ring order sigma, ring position p holds group sigma[p],
 *   which sends to sigma[p+1 mod G].  RNA: the fixed ring (identity,
 *   P_m -> P_{m+1}).  ARNA: a fresh Fisher-Yates shuffle of the identity at
 *   every step k >= 1, draw j from stream RING, index j, step k.
 * ORA_TOPO_NODE_RING (Sec. VI: neighbouring PEs of the ring on the same
 *   node): groups form nodes of node_groups consecutive groups (the last
 *   may be smaller).  ARNA: the ring visits the nodes in a shuffled order
 *   (Fisher-Yates over the nodes, draw j from RING call 1, index j) and each
 *   node's groups in a shuffled order (Fisher-Yates over its groups, draw j
 *   from RING call 2, index n node_groups + j), so only one ring edge per
 *   node leaves it.  RNA: the fixed ring, which is already node by node.
 * ORA_TOPO_HYPERCUBE (Sec. VI: another regular graph of low degree): at
 *   step k >= 1 every group g exchanges with its partner g xor 2^d (itself
 *   when that is >= G) along dimension d of the ceil(log2 G)-cube; RNA
 *   cycles d = (k - 1) mod D, ARNA draws d uniformly (RING call 3, index 0).
 *   sigma[g] is then g's partner.
 * At k = 0 (no exchange) and for G = 1 sigma is the identity. */
void ora_ring(const ora_cfg* c, uint32_t k, int32_t* sigma) {
  int32_t G = c->G;
  for (int32_t g = 0; g < G; ++g) sigma[g] = g;
  if (k == 0 || G == 1) return;
  if (c->topology == ORA_TOPO_HYPERCUBE) {
    int32_t D = ora_hyper_dims(G);
    uint32_t d = c->mode == ORA_ARNA ? draw_bounded_call(c, ORA_STREAM_RING, 3u, 0u, k, (uint32_t)D)
                                     : (k - 1u) % (uint32_t)D;
    for (int32_t g = 0; g < G; ++g) {
      int32_t p = g ^ (1 << d);
      sigma[g] = p < G ? p : g;
    }
    return;
  }
  if (c->mode != ORA_ARNA) return;
  if (c->topology == ORA_TOPO_NODE_RING) {
    int32_t B = c->node_groups < 1 ? 1 : c->node_groups;
    int32_t NN = (G + B - 1) / B;
    uint32_t* r = (uint32_t*)calloc((size_t)(NN > B ? NN : B), sizeof(uint32_t));
    int32_t* nodes = (int32_t*)malloc(sizeof(int32_t) * (size_t)NN);
    int32_t* members = (int32_t*)malloc(sizeof(int32_t) * (size_t)B);
    for (int32_t j = 1; j < NN; ++j) r[j] = draw_bounded_call(c, ORA_STREAM_RING, 1u, (uint32_t)j, k, (uint32_t)j + 1u);
    ora_fisher_yates(NN, r, nodes);
    int32_t pos = 0;
    for (int32_t q = 0; q < NN; ++q) {
      int32_t n = nodes[q], base = n * B, sz = (G - base < B) ? G - base : B;
      for (int32_t j = 1; j < sz; ++j)
        r[j] = draw_bounded_call(c, ORA_STREAM_RING, 2u, (uint32_t)(base + j), k, (uint32_t)j + 1u);
      ora_fisher_yates(sz, r, members);
      for (int32_t i = 0; i < sz; ++i) sigma[pos++] = base + members[i];
    }
    free(r);
    free(nodes);
    free(members);
    return;
  }
  uint32_t* r = (uint32_t*)calloc((size_t)G, sizeof(uint32_t));
  for (int32_t j = 1; j < G; ++j) r[j] = ora_draw_bounded(c, ORA_STREAM_RING, (uint32_t)j, k, (uint32_t)j + 1u);
  ora_fisher_yates(G, r, sigma);
  free(r);
}

/* pred[g]: the group that sends to g under ring order sigma. */
void ora_pred(int32_t G, const int32_t* sigma, int32_t* pred) {
  for (int32_t p = 0; p < G; ++p) pred[sigma[p]] = sigma[(p + G - 1) % G];
}

/* pred[g] for the track's topology: the ring's predecessor, or for the
 * hypercube the partner itself (the exchange is mutual). */
void ora_pred_topo(const ora_cfg* c, const int32_t* sigma, int32_t* pred) {
  if (c->topology == ORA_TOPO_HYPERCUBE)
    for (int32_t g = 0; g < c->G; ++g) pred[g] = sigma[g];
  else
    ora_pred(c->G, sigma, pred);
}

/* ------------------------------------------------------------------------ */
/* S2: exchange count (Eq. 3, Eq. 4; Sec. V-A cut-off).                     */
/* PE_eff is the effective number of groups, (sum W)^2 / sum W^2 over the    */
/* carried group weights W_m = exp(Lambda_m); it lies in [1, G].            */
/* ------------------------------------------------------------------------ */
double ora_pe_eff(int32_t G, const double* Lambda) {
  double mx = -INFINITY;
  for (int32_t m = 0; m < G; ++m)
    if (Lambda[m] > mx) mx = Lambda[m];
  if (!isfinite(mx)) return 0.0;
  double s = 0.0, s2 = 0.0;
  for (int32_t m = 0; m < G; ++m) {
    double w = exp(Lambda[m] - mx);
    s += w;
    s2 += w * w;
  }
  return s * s / s2;
}

int32_t ora_n_ex(const ora_cfg* c, uint32_t k, const double* Lambda, double* pe_eff_out) {
  int32_t G = c->G;
  double pe = ora_pe_eff(G, Lambda);
  if (pe_eff_out) *pe_eff_out = pe;
  if (k == 0 || G == 1) return 0;
  double rho;
  if (c->mode == ORA_ARNA) {
    if (!(pe < c->cutoff * (double)G)) {
      rho = 0.0;
    } else {
      rho = 0.5 - 0.5 * (pe - 1.0) / (double)(G - 1);
      if (rho < 0.0) rho = 0.0;
      if (rho > 0.5) rho = 0.5;
    }
  } else {
    rho = c->ex_ratio;
    if (rho < 0.0) rho = 0.0;
    if (rho > 1.0) rho = 1.0;
  }
  return (int32_t)floor(rho * (double)c->Np);
}

/* ------------------------------------------------------------------------ */
/* S3: local exchange with fixed group sizes (Sec. III-A, Sec. III-C).       */
/* Group g's send set at step k is the systematic slot subsample            */
/*   s_{g,t} = floor((t * Np + o_g) / N_ex),  t = 0 .. N_ex-1,               */
/* with o_g uniform in [0, Np) (stream EXCH, index g, step k); every slot is */
/* sent with probability N_ex / Np.  Group g's particle in slot s_{g,t}     */
/* moves to slot s_{r,t} of its successor r, carrying its origin weight.    */
/* ------------------------------------------------------------------------ */
uint32_t ora_exchange_offset(const ora_cfg* c, uint32_t g, uint32_t k) {
  return ora_draw_bounded(c, ORA_STREAM_EXCH, g, k, (uint32_t)c->Np);
}

/* ------------------------------------------------------------------------ */
/* Random send sets (Sec. III-C: each PE "randomly selects" the particles it */
/* sends), ORA_SEND_KEYED: group g's t-th sent slot at step k is             */
/* pi_g(t), t < N_ex, for a keyed pseudo-random permutation pi_g of [0, Np): */
/* a four-round Feistel network (Luby and Rackoff, SIAM J. Comput. 1988) on  */
/* b = ceil(log2 Np) bits, walked onto [0, Np) by repeating it while the     */
/* value is out of range (cycle walking: Black and Rogaway, "Ciphers with    */
/* arbitrary finite domains", CT-RSA 2002).  The b bits split into a high    */
/* half L of floor(b/2) bits and a low half R of the rest; a round maps      */
/* (L, R) to (R, L xor (F(R xor key_i) mod 2^|L|)), so the halves trade      */
/* places and sizes, and four rounds restore the sizes.  F is the mixer      */
/*   h = x * 0x9E3779B1; h ^= h >> 16; h *= 0x7FEB352D; h ^= h >> 15         */
/* (32-bit wrap-around).  key_0..3: the four Philox words of the EXCH stream, */
/* call 1, counter (g, 0, k).                                               */
/* ------------------------------------------------------------------------ */
static uint32_t feistel_mix(uint32_t x) {
  uint32_t h = x * 0x9E3779B1u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  return h;
}

static uint32_t low_mask(int n) { return n >= 32 ? 0xffffffffu : ((1u << n) - 1u); }

int ora_perm_bits(uint32_t n) {
  int b = 0;
  while (b < 32 && (1u << b) < n) ++b;
  return b;
}

static uint32_t feistel_fwd(uint32_t x, int b, const uint32_t key[4]) {
  int sl = b / 2, sr = b - sl;
  uint32_t L = x >> sr, R = x & low_mask(sr);
  for (int i = 0; i < 4; ++i) {
    uint32_t nl = R, nr = L ^ (feistel_mix(R ^ key[i]) & low_mask(sl));
    L = nl;
    R = nr;
    int t = sl; sl = sr; sr = t;
  }
  return (L << sr) | R;
}

static uint32_t feistel_inv(uint32_t y, int b, const uint32_t key[4]) {
  int sl = b / 2, sr = b - sl;
  uint32_t L = y >> sr, R = y & low_mask(sr);
  for (int i = 3; i >= 0; --i) {
    uint32_t nr = L, nl = R ^ (feistel_mix(L ^ key[i]) & low_mask(sr));
    L = nl;
    R = nr;
    int t = sl; sl = sr; sr = t;
  }
  return (L << sr) | R;
}

void ora_send_keys(const ora_cfg* c, uint32_t g, uint32_t k, uint32_t key[4]) {
  philox_stream(c, g, 0u, k, ORA_STREAM_EXCH, 1u, key);
}

uint32_t ora_send_perm(uint32_t t, uint32_t n, const uint32_t key[4]) {
  int b = ora_perm_bits(n);
  uint32_t x = t;
  do x = feistel_fwd(x, b, key); while (x >= n);
  return x;
}

uint32_t ora_send_perm_inv(uint32_t j, uint32_t n, const uint32_t key[4]) {
  int b = ora_perm_bits(n);
  uint32_t x = j;
  do x = feistel_inv(x, b, key); while (x >= n);
  return x;
}

/* S3: group pred(r) sends its t-th send slot (t < n_ex) to the t-th send
 * slot of r, pred from sigma as in ora_pred_topo (on a ring, sigma_p sends
 * to sigma_{p+1}).  Send slots: ORA_SEND_SYSTEMATIC, the systematic
 * subsample floor((t Np + o_g) / n_ex) with a uniform offset o_g in [0, Np);
 * ORA_SEND_KEYED, pi_g(t) of the keyed permutation above.
 * pop_in / pop_out: 5 x N SoA (component-major), N = G*Np, slot = g*Np + j.
 * src[i]: the slot that slot i's particle came from; origin[i]: its group. */
void ora_exchange(const ora_cfg* c, uint32_t k, const int32_t* sigma, int32_t n_ex,
                  const double* pop_in, double* pop_out, int32_t* src, int32_t* origin) {
  int32_t G = c->G, Np = c->Np;
  int64_t N = (int64_t)G * Np;
  for (int64_t i = 0; i < N; ++i) {
    src[i] = (int32_t)i;
    origin[i] = (int32_t)(i / Np);
  }
  if (n_ex > 0) {
    const int keyed = c->send_rule == ORA_SEND_KEYED;
    uint32_t* o = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)G);
    uint32_t* key = (uint32_t*)malloc(sizeof(uint32_t) * 4 * (size_t)G);
    for (int32_t g = 0; g < G; ++g) {
      o[g] = ora_exchange_offset(c, (uint32_t)g, k);
      ora_send_keys(c, (uint32_t)g, k, key + 4 * g);
    }
    int32_t* pred = (int32_t*)malloc(sizeof(int32_t) * (size_t)G);
    ora_pred_topo(c, sigma, pred);
    for (int32_t r = 0; r < G; ++r) {
      int32_t g = pred[r];
      for (int32_t t = 0; t < n_ex; ++t) {
        int64_t s_g = keyed ? (int64_t)ora_send_perm((uint32_t)t, (uint32_t)Np, key + 4 * g)
                            : ((int64_t)t * Np + o[g]) / n_ex;
        int64_t s_r = keyed ? (int64_t)ora_send_perm((uint32_t)t, (uint32_t)Np, key + 4 * r)
                            : ((int64_t)t * Np + o[r]) / n_ex;
        src[(int64_t)r * Np + s_r] = (int32_t)((int64_t)g * Np + s_g);
        origin[(int64_t)r * Np + s_r] = g;
      }
    }
    free(o);
    free(key);
    free(pred);
  }
  for (int d = 0; d < 5; ++d)
    for (int64_t i = 0; i < N; ++i) pop_out[d * N + i] = pop_in[d * N + src[i]];
}

/* ------------------------------------------------------------------------ */
/* S5: propagate (Alg. 1 step P) under nearly constant velocity (Sec. V),    */
/* unit frame interval, diagonal Gaussian process noise:                    */
/*   x += vx + s_pos e_x,  y += vy + s_pos e_y   (old velocity)              */
/*   vx += s_v e_vx,  vy += s_v e_vy,  I += s_I e_I.                          */
/* ------------------------------------------------------------------------ */
void ora_propagate(const ora_cfg* c, uint32_t k, const double* pop, double* X) {
  int32_t G = c->G, Np = c->Np;
  int64_t N = (int64_t)G * Np;
#pragma omp parallel for collapse(2) schedule(static) num_threads(ora_threads) if (ora_threads > 1)
  for (int32_t g = 0; g < G; ++g)
    for (int32_t j = 0; j < Np; ++j) {
      int64_t i = (int64_t)g * Np + j;
      double e[5];
      ora_normals(c, (uint32_t)g, (uint32_t)j, k, e);
      double x = pop[i], y = pop[N + i], vx = pop[2 * N + i], vy = pop[3 * N + i], I = pop[4 * N + i];
      X[i] = x + vx + c->sigma_pos * e[0];
      X[N + i] = y + vy + c->sigma_pos * e[1];
      X[2 * N + i] = vx + c->sigma_v * e[2];
      X[3 * N + i] = vy + c->sigma_v * e[3];
      X[4 * N + i] = I + c->sigma_I * e[4];
    }
}

/* ------------------------------------------------------------------------ */
/* S6: likelihood (Alg. 1 step U; Sec. V appearance model, Fig. 1).          */
/* A spot is a 2-D Gaussian of width sigma_psf and amplitude I on background */
/* b.  Over the (2R+1)^2 patch centred on the nearest pixel,                 */
/*   l = -sum (zbar - b - I gx(u) gy(v))^2 / (2 sigma_obs^2),                */
/* gx(u) = exp(-(u-x)^2 / (2 sigma_psf^2)); pixel (u,v) = (column,row) has   */
/* its centre at (u,v); zbar = z inside the image and b outside.            */
/* ------------------------------------------------------------------------ */
double ora_loglik_image(const ora_cfg* c, const float* frame, double x, double y, double I) {
  if (!isfinite(x) || !isfinite(y) || !isfinite(I)) return NAN;
  double cx = floor(x + 0.5), cy = floor(y + 0.5);
  double b = c->background, s2 = 2.0 * c->sigma_psf * c->sigma_psf;
  double acc = 0.0;
  for (int dv = -c->R; dv <= c->R; ++dv) {
    double v = cy + dv;
    for (int du = -c->R; du <= c->R; ++du) {
      double u = cx + du;
      double z = b;
      if (u >= 0.0 && u < (double)c->W && v >= 0.0 && v < (double)c->H)
        z = (double)frame[(int64_t)v * c->W + (int64_t)u];
      double gx = exp(-(u - x) * (u - x) / s2);
      double gy = exp(-(v - y) * (v - y) / s2);
      double r = z - b - I * gx * gy;
      acc += r * r;
    }
  }
  return -acc / (2.0 * c->sigma_obs * c->sigma_obs);
}

/* The Gaussian likelihood of the whole frame z_k (Sec. II's p(z_k | x_k))
 * with the spot model of ora_loglik_image (zero outside the patch), as a
 * ratio to the likelihood of the background alone: every pixel off the
 * patch contributes equally to both and cancels, leaving
 *   l = -sum_patch [ (zbar - b - I gx gy)^2 - (zbar - b)^2 ] / (2 sigma_obs^2).
 * Particles over plain background then score about 0 instead of the patch
 * residual of the noise alone. */
double ora_loglik_frame(const ora_cfg* c, const float* frame, double x, double y, double I) {
  if (!isfinite(x) || !isfinite(y) || !isfinite(I)) return NAN;
  double cx = floor(x + 0.5), cy = floor(y + 0.5);
  double b = c->background, s2 = 2.0 * c->sigma_psf * c->sigma_psf;
  double acc = 0.0;
  for (int dv = -c->R; dv <= c->R; ++dv) {
    double v = cy + dv;
    for (int du = -c->R; du <= c->R; ++du) {
      double u = cx + du;
      double z = b;
      if (u >= 0.0 && u < (double)c->W && v >= 0.0 && v < (double)c->H)
        z = (double)frame[(int64_t)v * c->W + (int64_t)u];
      double gx = exp(-(u - x) * (u - x) / s2);
      double gy = exp(-(v - y) * (v - y) / s2);
      double r = z - b - I * gx * gy;
      acc += r * r - (z - b) * (z - b);
    }
  }
  return -acc / (2.0 * c->sigma_obs * c->sigma_obs);
}

/* The image likelihood of c->obs_kind (ora_loglik_frame for ORA_OBS_FRAME,
 * else ora_loglik_image) for each column of a 5 x n state array. */
void ora_loglik_image_batch(const ora_cfg* c, const float* frame, const double* states, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = (c->obs_kind == ORA_OBS_FRAME) ? ora_loglik_frame(c, frame, states[i], states[n + i], states[4 * n + i])
                                            : ora_loglik_image(c, frame, states[i], states[n + i], states[4 * n + i]);
}

/* Linear-Gaussian observation of the position (z = (x, y) + noise), used
 * only to pin the filter against the Kalman filter. */
double ora_loglik_point(const ora_cfg* c, const float* obs, double x, double y) {
  double dx = x - (double)obs[0], dy = y - (double)obs[1];
  return -(dx * dx + dy * dy) / (2.0 * c->sigma_obs * c->sigma_obs);
}

/* ------------------------------------------------------------------------ */
/* S9 input: fixed-point weight codes, decided in FP32.                     */
/*   M = max lw (NaN ignored); t = fl(lw - M); z = fl(t * L2E);              */
/*   q = 0 if not (z >= -40);                                                */
/*   else n = rint(z), f = z - n (exact), p = Horner of sum_{d<=7} c_d f^d   */
/*   with c_d = fl32((ln 2)^d / d!) (built in FP64 as c_d = c_{d-1} ln2 / d, */
/*   FP32 fma at every step), q = trunc(p * 2^(n+40)).                      */
/* L2E = fl32(log2 e).  Every FP32 operation is a single correctly rounded  */
/* IEEE operation, so any machine gives the same q for the same lw.  q/2^40 */
/* approximates exp(lw - M) to about 2^-19 relative.                         */
/* ------------------------------------------------------------------------ */
static float ora_c[8];
static int ora_c_ready = 0;

static void ora_build_coeffs(void) {
  double d = 1.0;
  ora_c[0] = 1.0f;
  for (int k = 1; k < 8; ++k) {
    d = d * ORA_LN2 / (double)k;
    ora_c[k] = (float)d;
  }
  ora_c_ready = 1;
}

void ora_exp2_coeffs(float out[8]) {
  if (!ora_c_ready) ora_build_coeffs();
  memcpy(out, ora_c, sizeof(ora_c));
}

static uint64_t quantize_one(float lw, float M) {
  const float L2E = (float)1.4426950408889634;
  float t = lw - M;
  float z = t * L2E;
  if (!(z >= -40.0f)) return 0;
  float n = rintf(z);
  float f = z - n;
  float p = ora_c[7];
  for (int d = 6; d >= 0; --d) p = fmaf(p, f, ora_c[d]);
  float v = ldexpf(p, (int)n + 40);
  return (uint64_t)v;
}

void ora_quantize(const float* lw, int32_t n, uint64_t* q) {
  if (!ora_c_ready) ora_build_coeffs();
  float M = -INFINITY;
  for (int32_t i = 0; i < n; ++i) M = fmaxf(M, lw[i]);
  for (int32_t i = 0; i < n; ++i) q[i] = quantize_one(lw[i], M);
}

/* ------------------------------------------------------------------------ */
/* S9: systematic resampling (Alg. 1 step 6; Alg. 2/3 "resample"), exact.    */
/* With Q = sum q, S_i = sum_{l<i} q_l and phi = u / 2^32, output j takes    */
/* the particle i with S_i <= (j + phi) Q / n < S_{i+1}; in integers:        */
/*   anc[j] = min{ i : (j 2^32 + u) Q < S_{i+1} n 2^32 }.                    */
/* This is the textbook two-pointer sweep with exact 128-bit comparisons.    */
/* Q = 0 (a group with no finite weight) resamples as the identity.          */
/* ------------------------------------------------------------------------ */
void ora_resample(const uint64_t* q, int32_t n, uint32_t u, int32_t* anc) {
  u128 Q = 0;
  for (int32_t i = 0; i < n; ++i) Q += q[i];
  if (Q == 0) {
    for (int32_t j = 0; j < n; ++j) anc[j] = j;
    return;
  }
  int32_t i = 0;
  u128 S_next = q[0];
  for (int32_t j = 0; j < n; ++j) {
    u128 lhs = ((((u128)j) << 32) | (u128)u) * Q;
    while (!(lhs < ((S_next * (u128)n) << 32))) {
      ++i;
      S_next += q[i];
    }
    anc[j] = i;
  }
}

uint32_t ora_resample_uniform(const ora_cfg* c, uint32_t g, uint32_t k) {
  uint32_t w[4];
  philox_stream(c, g, 0u, k, ORA_STREAM_RESAMPLE, 0u, w);
  return w[0];
}

/* ------------------------------------------------------------------------ */
/* Alg. 1's resampling test, per group: resample when the effective sample  */
/* size N_eff = 1 / sum_i w_i^2 of the normalised weights falls below       */
/* N_thresh (Sec. II: when too few particles carry relatively high weight). */
/* Taken on the resampler's weight codes so that both sides decide alike:   */
/* w_i = c_i / sum c with c_i = q_i >> 20 (in [0, 2^20]), so               */
/* N_eff = (sum c)^2 / sum c^2; N_thresh = t Np / 2^16 with                 */
/* t = round(ess_fraction 2^16).  In exact integers:                        */
/*   resample  iff  2^16 (sum c)^2 < t Np sum c^2.                          */
/* Returns 1 to resample.  Q = 0 (no finite weight) returns 1: such a group */
/* resamples as the identity.                                               */
/* ------------------------------------------------------------------------ */
uint32_t ora_ess_code(double ess_fraction) {
  double f = ess_fraction < 0.0 ? 0.0 : (ess_fraction > 1.0 ? 1.0 : ess_fraction);
  return (uint32_t)floor(f * 65536.0 + 0.5);
}

int ora_ess_test(const uint64_t* q, int32_t n, double ess_fraction) {
  u128 Q = 0, s1 = 0, s2 = 0;
  for (int32_t i = 0; i < n; ++i) {
    uint64_t c = q[i] >> 20;
    Q += q[i];
    s1 += c;
    s2 += (u128)c * c;
  }
  if (Q == 0) return 1;
  u128 t = ora_ess_code(ess_fraction);
  return ((s1 * s1) << 16) < t * (u128)n * s2;
}

/* ------------------------------------------------------------------------ */
/* Initial population (Sec. V "tracking" and "information sharing" modes).  */
/* INIT stream, index j, group g, step 0: call 0 words 0..3, call 1 word 0.  */
/*  POINT:    every particle at x0.                                          */
/*  UNIFORM:  component d uniform in [lo_d, hi_d].                           */
/*  SHARING:  group 0 at x0 with the position uniform in the disc of radius  */
/*            `radius` (r = radius sqrt(u0), angle 2 pi u1); other groups    */
/*            UNIFORM.                                                      */
/* ------------------------------------------------------------------------ */
void ora_init(const ora_cfg* c, int32_t kind, const double* x0, const double* lo, const double* hi,
              double radius, double* pop) {
  int32_t G = c->G, Np = c->Np;
  int64_t N = (int64_t)G * Np;
  for (int32_t g = 0; g < G; ++g)
    for (int32_t j = 0; j < Np; ++j) {
      int64_t i = (int64_t)g * Np + j;
      uint32_t a[4], b[4];
      philox_stream(c, (uint32_t)j, (uint32_t)g, 0u, ORA_STREAM_INIT, 0u, a);
      philox_stream(c, (uint32_t)j, (uint32_t)g, 0u, ORA_STREAM_INIT, 1u, b);
      double u[5] = {ora_uniform(a[0]), ora_uniform(a[1]), ora_uniform(a[2]), ora_uniform(a[3]),
                     ora_uniform(b[0])};
      double s[5];
      if (kind == ORA_INIT_POINT || (kind == ORA_INIT_SHARING && g == 0)) {
        for (int d = 0; d < 5; ++d) s[d] = x0[d];
        if (kind == ORA_INIT_SHARING) {
          double r = radius * sqrt(u[0]), th = 2.0 * ORA_PI * u[1];
          s[0] = x0[0] + r * cos(th);
          s[1] = x0[1] + r * sin(th);
        }
      } else {
        for (int d = 0; d < 5; ++d) s[d] = lo[d] + (hi[d] - lo[d]) * u[d];
      }
      for (int d = 0; d < 5; ++d) pop[d * N + i] = s[d];
    }
}

/* ------------------------------------------------------------------------ */
/* One step k of Alg. 3 (ARNA) / Alg. 2 (RNA) for one track.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* all arrays caller-allocated; N = G*Np */
  int32_t* sigma;     /* [G]   S1 ring order */
  int32_t* n_ex;      /* [1]   S2 */
  double* pe_eff;     /* [1]   S2, from Lambda_in */
  int32_t* src;       /* [N]   S3 slot map */
  int32_t* origin;    /* [N]   S3 origin group */
  double* X;          /* [5N]  S5 propagated states (SoA) */
  double* loglik;     /* [N]   S6 l_i */
  double* lw;         /* [N]   S4+S6 log w~_i = log w_i + l_i */
  uint64_t* q;        /* [N]   S9 weight codes */
  int32_t* anc;       /* [N]   S9 ancestors (slot within the group) */
  double* Lambda_out; /* [G]   S7/S10 group log-weights Lambda'_m */
  double* gxhat;      /* [5G]  S7 group estimates xhat^m (SoA: d*G + m) */
  double* gess;       /* [G]   S7 group ESS */
  double* logc;       /* [1]   S8 log of the incremental likelihood */
  double* xhat;       /* [5]   S8 global estimate */
  double* pop_out;    /* [5N]  resampled population (input of step k+1) */
  int32_t* degenerate;/* [1]   groups with no finite weight */
  double* omega;      /* [N]   log of each output slot's weight within its group (S10) */
  int32_t* resampled; /* [G]   1 where the group resampled at this step */
} ora_step_out;

static double lse(const double* v, int64_t n) {
  double mx = -INFINITY;
  for (int64_t i = 0; i < n; ++i)
    if (v[i] > mx) mx = v[i];
  if (!isfinite(mx)) return mx;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += exp(v[i] - mx);
  return mx + log(s);
}

/* pop_in: the population after step k-1's resampling (5 x N, SoA), the
 * particle in slot i of group m carrying weight W_m w_i with
 * W_m = exp(Lambda_in[m]) and w_i = exp(omega_in[i]) its weight within the
 * group (Alg. 3 step 8: w_i = 1 / Np after resampling; omega_in may then be
 * NULL).  A group that skipped resampling under ORA_RESAMPLE_ESS carries its
 * particles' own normalised weights instead.  At k = 0 pop_in is the initial
 * sample, Lambda_in and omega_in are ignored (all weights equal).  obs: the frame (H x W, row-major) or, for
 * ORA_OBS_POINT, two floats.  lw_override: if not NULL, steps S7-S9 (group
 * weights, estimates, resampling) use these FP32 log-weights instead of the
 * oracle's own (so both sides can be fed identical weights); o->lw still
 * receives the oracle's own.  Returns 0, or 1 if every group is degenerate. */
int ora_step(const ora_cfg* c, uint32_t k, const float* obs, const double* pop_in,
             const double* Lambda_in, const double* omega_in, const float* lw_override, ora_step_out* o) {
  int32_t G = c->G, Np = c->Np;
  int64_t N = (int64_t)G * Np;
  double* Lam = (double*)malloc(sizeof(double) * (size_t)G);
  for (int32_t m = 0; m < G; ++m) Lam[m] = (k == 0) ? 0.0 : Lambda_in[m];

  /* S1, S2 (Alg. 3 steps 1-2) */
  ora_ring(c, k, o->sigma);
  *o->n_ex = ora_n_ex(c, k, Lam, o->pe_eff);

  /* S3 (Alg. 3 step 3) */
  double* pop = (double*)malloc(sizeof(double) * (size_t)(5 * N));
  ora_exchange(c, k, o->sigma, *o->n_ex, pop_in, pop, o->src, o->origin);

  /* S4 (Alg. 3 step 4): log w_i = Lambda_origin + omega_i - LSE(Lambda),
   * omega_i = -log Np after resampling; an exchanged particle keeps its own */
  double lse_lam = lse(Lam, G);
  double* om = (double*)malloc(sizeof(double) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) om[i] = (k == 0 || !omega_in) ? -log((double)Np) : omega_in[o->src[i]];

  /* S5, S6 (Alg. 3 step 5) */
  if (k == 0)
    memcpy(o->X, pop, sizeof(double) * (size_t)(5 * N));
  else
    ora_propagate(c, k, pop, o->X);
#pragma omp parallel for schedule(static) num_threads(ora_threads) if (ora_threads > 1)
  for (int64_t i = 0; i < N; ++i) {
    double x = o->X[i], y = o->X[N + i], I = o->X[4 * N + i];
    double l = (c->obs_kind == ORA_OBS_POINT)   ? ora_loglik_point(c, obs, x, y)
               : (c->obs_kind == ORA_OBS_FRAME) ? ora_loglik_frame(c, obs, x, y, I)
                                                : ora_loglik_image(c, obs, x, y, I);
    o->loglik[i] = l;
    o->lw[i] = Lam[o->origin[i]] + om[i] - lse_lam + l;
  }

  /* With lw_override the remaining steps (S7-S9) use those log-weights, so
   * that both sides can be fed identical weights. */
  double* lwe = o->lw;
  double* lwbuf = NULL;
  if (lw_override) {
    lwbuf = (double*)malloc(sizeof(double) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) lwbuf[i] = (double)lw_override[i];
    lwe = lwbuf;
  }

  /* S7 (Alg. 3 step 6): group estimate and group weight, FP64 */
  int32_t degen = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : degen) num_threads(ora_threads) if (ora_threads > 1)
  for (int32_t m = 0; m < G; ++m) {
    const double* lwm = lwe + (int64_t)m * Np;
    double mx = -INFINITY;
    for (int32_t j = 0; j < Np; ++j)
      if (lwm[j] > mx) mx = lwm[j];
    double s = 0.0, s2 = 0.0, sx[5] = {0, 0, 0, 0, 0};
    if (isfinite(mx)) {
      for (int32_t j = 0; j < Np; ++j) {
        double w = isnan(lwm[j]) ? 0.0 : exp(lwm[j] - mx);
        s += w;
        s2 += w * w;
        for (int d = 0; d < 5; ++d) sx[d] += w * o->X[d * N + (int64_t)m * Np + j];
      }
      o->Lambda_out[m] = mx + log(s);
      for (int d = 0; d < 5; ++d) o->gxhat[d * G + m] = sx[d] / s;
      o->gess[m] = s * s / s2;
    } else {
      ++degen;
      o->Lambda_out[m] = -INFINITY;
      for (int d = 0; d < 5; ++d) o->gxhat[d * G + m] = 0.0;
      o->gess[m] = 0.0;
    }
  }
  *o->degenerate = degen;

  /* S8 (Alg. 3 steps 9-10): the master's reduction */
  *o->logc = lse(o->Lambda_out, G);
  for (int d = 0; d < 5; ++d) {
    double acc = 0.0;
    if (isfinite(*o->logc))
      for (int32_t m = 0; m < G; ++m)
        if (isfinite(o->Lambda_out[m])) acc += exp(o->Lambda_out[m] - *o->logc) * o->gxhat[d * G + m];
    o->xhat[d] = acc;
  }

  /* S9 (Alg. 3 step 7): per-group systematic resampling on FP32 codes; under
   * ORA_RESAMPLE_ESS only where Alg. 1's N_eff test asks for it.  S10: a
   * resampled group's particles weigh 1 / Np within it, the others keep
   * w_i = w~_i / W'_m. */
  ora_build_coeffs(); /* the weight-code table, before any thread uses it */
#pragma omp parallel for schedule(dynamic, 1) num_threads(ora_threads) if (ora_threads > 1)
  for (int32_t m = 0; m < G; ++m) {
    float* lwf = (float*)malloc(sizeof(float) * (size_t)Np);
    for (int32_t j = 0; j < Np; ++j)
      lwf[j] = lw_override ? lw_override[(int64_t)m * Np + j] : (float)o->lw[(int64_t)m * Np + j];
    uint64_t* qm = o->q + (int64_t)m * Np;
    int32_t* am = o->anc + (int64_t)m * Np;
    double* omm = o->omega + (int64_t)m * Np;
    ora_quantize(lwf, Np, qm);
    int res = c->resample_rule != ORA_RESAMPLE_ESS || ora_ess_test(qm, Np, c->ess_fraction);
    o->resampled[m] = res;
    if (res) {
      ora_resample(qm, Np, ora_resample_uniform(c, (uint32_t)m, k), am);
      for (int32_t j = 0; j < Np; ++j) omm[j] = -log((double)Np);
    } else {
      for (int32_t j = 0; j < Np; ++j) {
        am[j] = j;
        omm[j] = lwe[(int64_t)m * Np + j] - o->Lambda_out[m];
      }
    }
    free(lwf);
  }
  free(lwbuf);
  free(om);

  /* S10 (Alg. 3 step 8): the resampled population; group weights carried */
#pragma omp parallel for collapse(2) schedule(static) num_threads(ora_threads) if (ora_threads > 1)
  for (int d = 0; d < 5; ++d)
    for (int32_t m = 0; m < G; ++m)
      for (int32_t j = 0; j < Np; ++j) {
        int64_t i = (int64_t)m * Np + j;
        o->pop_out[d * N + i] = o->X[d * N + (int64_t)m * Np + o->anc[i]];
      }

  free(pop);
  free(Lam);
  return degen == G ? 1 : 0;
}

/* A whole run of T steps from the initial population pop0 (5 x N).
 * Per-step outputs (caller-allocated, step-major): xhat[T*5], logc[T],
 * n_ex[T], pe_eff[T], sigma[T*G], Lambda[T*G], gxhat[T*5*G], n_resampled[T]
 * (groups that resampled).  Any per-step pointer may be NULL.  obs: T frames (H*W floats each) or T points (2
 * floats each).  Returns the first step at which every group was degenerate,
 * or -1. */
int ora_run(const ora_cfg* c, const double* pop0, const float* obs, int32_t T, double* xhat,
            double* logc, int32_t* n_ex, double* pe_eff, int32_t* sigma, double* Lambda,
            double* gxhat, int32_t* n_resampled, double* pop_final) {
  int32_t G = c->G, Np = c->Np;
  int64_t N = (int64_t)G * Np;
  size_t fs = (c->obs_kind == ORA_OBS_POINT) ? 2 : (size_t)c->H * (size_t)c->W;
  double* pop = (double*)malloc(sizeof(double) * (size_t)(5 * N));
  double* Lam = (double*)calloc((size_t)G, sizeof(double));
  memcpy(pop, pop0, sizeof(double) * (size_t)(5 * N));
  ora_step_out o;
  o.sigma = (int32_t*)malloc(sizeof(int32_t) * (size_t)G);
  o.n_ex = (int32_t*)malloc(sizeof(int32_t));
  o.pe_eff = (double*)malloc(sizeof(double));
  o.src = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  o.origin = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  o.X = (double*)malloc(sizeof(double) * (size_t)(5 * N));
  o.loglik = (double*)malloc(sizeof(double) * (size_t)N);
  o.lw = (double*)malloc(sizeof(double) * (size_t)N);
  o.q = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
  o.anc = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  o.Lambda_out = (double*)malloc(sizeof(double) * (size_t)G);
  o.gxhat = (double*)malloc(sizeof(double) * (size_t)(5 * G));
  o.gess = (double*)malloc(sizeof(double) * (size_t)G);
  o.logc = (double*)malloc(sizeof(double));
  o.xhat = (double*)malloc(sizeof(double) * 5);
  o.pop_out = (double*)malloc(sizeof(double) * (size_t)(5 * N));
  o.degenerate = (int32_t*)malloc(sizeof(int32_t));
  o.omega = (double*)malloc(sizeof(double) * (size_t)N);
  o.resampled = (int32_t*)malloc(sizeof(int32_t) * (size_t)G);
  double* omega = (double*)malloc(sizeof(double) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) omega[i] = -log((double)Np);
  int failed = -1;
  for (int32_t k = 0; k < T; ++k) {
    int rc = ora_step(c, (uint32_t)k, obs + (size_t)k * fs, pop, Lam, omega, NULL, &o);
    if (rc && failed < 0) failed = k;
    if (xhat) memcpy(xhat + (size_t)k * 5, o.xhat, sizeof(double) * 5);
    if (logc) logc[k] = *o.logc;
    if (n_ex) n_ex[k] = *o.n_ex;
    if (pe_eff) pe_eff[k] = *o.pe_eff;
    if (sigma) memcpy(sigma + (size_t)k * G, o.sigma, sizeof(int32_t) * (size_t)G);
    if (Lambda) memcpy(Lambda + (size_t)k * G, o.Lambda_out, sizeof(double) * (size_t)G);
    if (gxhat) memcpy(gxhat + (size_t)k * 5 * G, o.gxhat, sizeof(double) * (size_t)(5 * G));
    if (n_resampled) {
      n_resampled[k] = 0;
      for (int32_t m = 0; m < G; ++m) n_resampled[k] += o.resampled[m];
    }
    memcpy(Lam, o.Lambda_out, sizeof(double) * (size_t)G);
    memcpy(omega, o.omega, sizeof(double) * (size_t)N);
    memcpy(pop, o.pop_out, sizeof(double) * (size_t)(5 * N));
  }
  if (pop_final) memcpy(pop_final, pop, sizeof(double) * (size_t)(5 * N));
  free(o.sigma); free(o.n_ex); free(o.pe_eff); free(o.src); free(o.origin); free(o.X);
  free(o.loglik); free(o.lw); free(o.q); free(o.anc); free(o.Lambda_out); free(o.gxhat);
  free(o.gess); free(o.logc); free(o.xhat); free(o.pop_out); free(o.degenerate);
  free(o.omega); free(o.resampled); free(omega);
  free(pop);
  free(Lam);
  return failed;
}

/* ------------------------------------------------------------------------ */
/* Gradient of log Z with respect to theta = (sigma_psf, A, b, sigma_pos,   */
/* sigma_v) with the resampling ancestry frozen.                             */
/* ------------------------------------------------------------------------ */

/* l of ora_loglik_image (ora_loglik_frame when obs_kind is ORA_OBS_FRAME)
 * and its partial derivatives with respect to x, y, I (state) and
 * sigma_psf, b (parameters): d[0..4] = dl/dx, dl/dy, dl/dI, dl/dsigma_psf,
 * dl/db.  The patch centre is piecewise constant in the state, so it
 * contributes no derivative.  Pixels outside the image read b, so their
 * residual does not depend on b.  The frame model's extra term
 * (zbar - b)^2 depends on b only. */
double ora_loglik_image_grad(const ora_cfg* c, const float* frame, double x, double y, double I, double d[5]) {
  for (int q = 0; q < 5; ++q) d[q] = 0.0;
  if (!isfinite(x) || !isfinite(y) || !isfinite(I)) return NAN;
  double cx = floor(x + 0.5), cy = floor(y + 0.5);
  double b = c->background, s = c->sigma_psf, s2 = 2.0 * s * s, so2 = c->sigma_obs * c->sigma_obs;
  double acc = 0.0;
  for (int dv = -c->R; dv <= c->R; ++dv) {
    double v = cy + dv;
    for (int du = -c->R; du <= c->R; ++du) {
      double u = cx + du;
      int inside = (u >= 0.0 && u < (double)c->W && v >= 0.0 && v < (double)c->H);
      double z = inside ? (double)frame[(int64_t)v * c->W + (int64_t)u] : b;
      double gx = exp(-(u - x) * (u - x) / s2);
      double gy = exp(-(v - y) * (v - y) / s2);
      double m = I * gx * gy;
      double r = z - b - m;
      acc += r * r;
      if (c->obs_kind == ORA_OBS_FRAME) {
        acc -= (z - b) * (z - b);
        if (inside) d[4] -= z - b;
      }
      /* dl/dtheta = -(1/so2) sum r dr/dtheta, dr/dtheta = -dm/dtheta (and -1 for b inside) */
      d[0] += r * m * (u - x) / (s * s);
      d[1] += r * m * (v - y) / (s * s);
      d[2] += r * gx * gy;
      d[3] += r * m * ((u - x) * (u - x) + (v - y) * (v - y)) / (s * s * s);
      if (inside) d[4] += r;
    }
  }
  for (int q = 0; q < 5; ++q) d[q] /= so2;
  return -acc / (2.0 * so2);
}

/* Replay of steps 0 .. T-1 with frozen ancestry, FP64, with forward-mode
 * tangents.  parents: T rows of N track-local slots; row k (k >= 1) gives
 * the slot of X_{k-1} each slot of step k was propagated from (the exchange
 * composed with the previous resampling), so its origin group is
 * parent / Np; row 0 is not read.  The initial population is drawn as in
 * ora_init with theta's A as the initial intensity (POINT: every particle;
 * SHARING: group 0).  Writes log Z = sum_k log c_k and grad[5] = d log Z /
 * d theta.  Per step (Alg. 3): X_k = NCV(X_{k-1}[parent]) (k >= 1),
 * lw = Lambda_bar_{k-1}[origin] - log Np + l, Lambda_k,m = LSE_{i in m} lw,
 * log c_k = LSE_m Lambda_k,m, Lambda_bar_k = Lambda_k - log c_k. */
/* round_f32: 0 for the FP64 replay; 1 to hold the states in FP32 (each state
 * component rounded to the nearest float after the initial draw and after
 * every propagation, everything else in FP64).  The second form measures how
 * far the estimator moves when only its states are stored in FP32, as a GPU
 * filter with FP32 states stores them: the patch centre of a particle that
 * sits within a rounding of a half-pixel boundary can change, and log Z is
 * discontinuous there.
 * states: NULL, or T x 5 x N given states (SoA per step); the replay then
 * takes step k's states from states[k] instead of computing them (the
 * tangents still follow the ancestry and the noise), so that the likelihood
 * and its derivatives are evaluated at exactly those states -- for
 * instance the states of an implementation under test, which removes the
 * difference its own state arithmetic makes and leaves that of its
 * gradient. */
int ora_replay_grad_ex(const ora_cfg* c, int32_t kind, const double* x0, const double* lo, const double* hi,
                       double radius, const float* frames, int32_t T, const int32_t* parents, int32_t round_f32,
                       const double* states, double* logZ, double* grad) {
  /* every step resamples here: a replay does not carry per-particle weights */
  if (c->resample_rule != ORA_RESAMPLE_ALWAYS) return -1;
  int32_t G = c->G, Np = c->Np;
  int64_t N = (int64_t)G * Np;
  size_t fs = (size_t)c->H * (size_t)c->W;
  double* X = (double*)malloc(sizeof(double) * (size_t)(5 * N));
  double* Xn = (double*)malloc(sizeof(double) * (size_t)(5 * N));
  double* dX = (double*)calloc((size_t)(25 * N), sizeof(double)); /* dX[(i*5 + d)*5 + p] */
  double* dXn = (double*)calloc((size_t)(25 * N), sizeof(double));
  double* lw = (double*)malloc(sizeof(double) * (size_t)N);
  double* dlw = (double*)malloc(sizeof(double) * (size_t)(5 * N));
  double* lbar = (double*)malloc(sizeof(double) * (size_t)G);
  double* dlbar = (double*)calloc((size_t)(5 * G), sizeof(double));
  double* Lam = (double*)malloc(sizeof(double) * (size_t)G);
  double* dLam = (double*)malloc(sizeof(double) * (size_t)(5 * G));
  ora_init(c, kind, x0, lo, hi, radius, X);
  if (round_f32)
    for (int64_t i = 0; i < 5 * N; ++i) X[i] = (double)(float)X[i];
  if (states) memcpy(X, states, sizeof(double) * (size_t)(5 * N));
  if (kind == ORA_INIT_POINT || kind == ORA_INIT_SHARING)
    for (int64_t i = 0; i < N; ++i)
      if (kind == ORA_INIT_POINT || i < Np) dX[(i * 5 + 4) * 5 + 1] = 1.0; /* dI/dA */
  for (int32_t m = 0; m < G; ++m) lbar[m] = -log((double)G);
  double lz = 0.0, gz[5] = {0, 0, 0, 0, 0};
  for (int32_t k = 0; k < T; ++k) {
    if (k >= 1) {
      const int32_t* par = parents + (int64_t)k * N;
#pragma omp parallel for collapse(2) schedule(static) num_threads(ora_threads) if (ora_threads > 1)
      for (int32_t g = 0; g < G; ++g)
        for (int32_t j = 0; j < Np; ++j) {
          int64_t i = (int64_t)g * Np + j, p = par[i];
          double e[5];
          ora_normals(c, (uint32_t)g, (uint32_t)j, (uint32_t)k, e);
          Xn[i] = X[p] + X[2 * N + p] + c->sigma_pos * e[0];
          Xn[N + i] = X[N + p] + X[3 * N + p] + c->sigma_pos * e[1];
          Xn[2 * N + i] = X[2 * N + p] + c->sigma_v * e[2];
          Xn[3 * N + i] = X[3 * N + p] + c->sigma_v * e[3];
          Xn[4 * N + i] = X[4 * N + p] + c->sigma_I * e[4];
          for (int q = 0; q < 5; ++q) {
            double px = dX[(p * 5 + 0) * 5 + q], py = dX[(p * 5 + 1) * 5 + q];
            double pvx = dX[(p * 5 + 2) * 5 + q], pvy = dX[(p * 5 + 3) * 5 + q];
            double pI = dX[(p * 5 + 4) * 5 + q];
            dXn[(i * 5 + 0) * 5 + q] = px + pvx + (q == 3 ? e[0] : 0.0);
            dXn[(i * 5 + 1) * 5 + q] = py + pvy + (q == 3 ? e[1] : 0.0);
            dXn[(i * 5 + 2) * 5 + q] = pvx + (q == 4 ? e[2] : 0.0);
            dXn[(i * 5 + 3) * 5 + q] = pvy + (q == 4 ? e[3] : 0.0);
            dXn[(i * 5 + 4) * 5 + q] = pI;
          }
        }
      double* t = X; X = Xn; Xn = t;
      t = dX; dX = dXn; dXn = t;
      if (round_f32)
        for (int64_t i = 0; i < 5 * N; ++i) X[i] = (double)(float)X[i];
      if (states) memcpy(X, states + (size_t)k * (size_t)(5 * N), sizeof(double) * (size_t)(5 * N));
    }
    /* weights and their tangents */
#pragma omp parallel for schedule(static) num_threads(ora_threads) if (ora_threads > 1)
    for (int64_t i = 0; i < N; ++i) {
      int32_t o = (k == 0) ? (int32_t)(i / Np) : (int32_t)(parents[(int64_t)k * N + i] / Np);
      double dl[5];
      double l = ora_loglik_image_grad(c, frames + (size_t)k * fs, X[i], X[N + i], X[4 * N + i], dl);
      lw[i] = lbar[o] - log((double)Np) + l;
      for (int q = 0; q < 5; ++q) {
        double v = dl[0] * dX[(i * 5 + 0) * 5 + q] + dl[1] * dX[(i * 5 + 1) * 5 + q] +
                   dl[2] * dX[(i * 5 + 4) * 5 + q];
        if (q == 0) v += dl[3];
        if (q == 2) v += dl[4];
        dlw[i * 5 + q] = dlbar[o * 5 + q] + v;
      }
    }
    for (int32_t m = 0; m < G; ++m) {
      const double* lm = lw + (int64_t)m * Np;
      double mx = -INFINITY;
      for (int32_t j = 0; j < Np; ++j)
        if (lm[j] > mx) mx = lm[j];
      double s = 0.0, ds[5] = {0, 0, 0, 0, 0};
      for (int32_t j = 0; j < Np; ++j) {
        double w = exp(lm[j] - mx);
        s += w;
        for (int q = 0; q < 5; ++q) ds[q] += w * dlw[((int64_t)m * Np + j) * 5 + q];
      }
      Lam[m] = mx + log(s);
      for (int q = 0; q < 5; ++q) dLam[m * 5 + q] = ds[q] / s;
    }
    double lc = lse(Lam, G), dlc[5] = {0, 0, 0, 0, 0};
    for (int32_t m = 0; m < G; ++m) {
      double pi = exp(Lam[m] - lc);
      for (int q = 0; q < 5; ++q) dlc[q] += pi * dLam[m * 5 + q];
    }
    lz += lc;
    for (int q = 0; q < 5; ++q) gz[q] += dlc[q];
    for (int32_t m = 0; m < G; ++m) {
      lbar[m] = Lam[m] - lc;
      for (int q = 0; q < 5; ++q) dlbar[m * 5 + q] = dLam[m * 5 + q] - dlc[q];
    }
  }
  *logZ = lz;
  for (int q = 0; q < 5; ++q) grad[q] = gz[q];
  free(X); free(Xn); free(dX); free(dXn); free(lw); free(dlw); free(lbar); free(dlbar); free(Lam); free(dLam);
  return 0;
}

/* The FP64 replay (ora_replay_grad_ex with round_f32 = 0). */
int ora_replay_grad(const ora_cfg* c, int32_t kind, const double* x0, const double* lo, const double* hi,
                    double radius, const float* frames, int32_t T, const int32_t* parents, double* logZ,
                    double* grad) {
  return ora_replay_grad_ex(c, kind, x0, lo, hi, radius, frames, T, parents, 0, NULL, logZ, grad);
}
