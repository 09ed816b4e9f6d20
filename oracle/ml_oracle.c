/*
 * ml_oracle.c -- plain, slow FP64 CPU oracle for the Luescher-Weisz multilevel
 * Monte Carlo of d=3+1 compact U(1) Wilson-action lattice gauge theory, as used
 * by Amado, Cardoso & Bicudo, "Flux tube widening in compact U(1) lattice gauge
 * theory computed at T < T_c with the multilevel method and GPUs"
 * (arXiv:1309.3859).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA implementation; it has its own Philox
 * generator, its own von Mises sampler and its own observables, written from
 * the paper (and, where the paper is silent, from the published algorithms
 * named below).
 *
 * Everything is double precision.  The code follows the method's steps in the
 * paper's order with no blocking, fusion or reordering beyond what the
 * definitions state.  The link-update loop of one (direction, parity) pass may
 * run under OpenMP: the links of one pass share no plaquette, so the order in
 * which they are visited does not change the result.  Every sum over sites
 * is serial, so the oracle is deterministic for any thread count.
 *
 * Conventions (shared with the CUDA path only through their published
 * definitions, restated here):
 *   site index    i = x + L*(y + L*(z + L*t)), periodic in all directions
 *   direction     0 = t (the paper's U_0), 1 = x, 2 = y, 3 = z
 *   angles        theta[mu*V + i], U_mu(i) = exp(i*theta), kept in [-pi, pi)
 *   parity        (x + y + z + t) mod 2
 *
 * Parity pins (tests/test_oracle_*.py): Philox known-answer vectors, the
 * chi-squared of the von Mises sampler against its density, overrelaxation
 * invariants, the strong-coupling plaquette I1(beta)/I0(beta), gauge
 * invariance, beta = 0 means, the n2 = 1 multilevel identity, multilevel
 * versus naive P(r), and the vanishing of <P> and Im P+P.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_TWO_PI (2.0 * ORC_PI)
#define ORC_MAX_TRIALS 64

/* Status codes returned by the oracle entry points. */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_EREJECT -5

typedef struct {
  int L, Nt;
  double beta;
  uint64_t seed;
  int n_or;        /* overrelaxation sweeps per heatbath sweep (Section II: 3) */
  int draws;       /* 0: 52-bit uniforms, two Philox blocks per trial;
                      1: 23-bit uniforms, two trials per Philox block        */
  int slab;        /* inner slab thickness d                                 */
  int n_sub;       /* inner sub-updates n2 (Algorithm 1)                     */
  int outer_slab;  /* 0 = single level, else outer slab thickness (Alg. 1: 4) */
  int n_sub_outer; /* outer sub-updates n4                                   */
  int k_between;   /* full compound sweeps before each measurement, k0       */
  int nr;
  const int *r;    /* P(r) separations                                       */
  int nrf;
  const int *rf;   /* separations of the field profile                       */
  int nprobe;
  const int *probe_dy, *probe_dz; /* transverse probe offsets                */
  unsigned comp_mask; /* bit c set: component c of (Ex,Ey,Ez,Bx,By,Bz)       */
  int threads;     /* OpenMP threads for link updates, 0 = runtime default   */
  int update;      /* update of the first sweep of a compound sweep:
                      0 heatbath, 1 Metropolis (Section II)                  */
  int metro_hits;  /* Metropolis hits per link visit                         */
  double metro_width; /* Metropolis proposal half-width w (radians)          */
  int multihit;    /* 1: P(r) at r >= 2 from the analytic multihit of the
                      temporal links (Section II.C)                          */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator: Salmon, Moraes, Dror & Shaw,       */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11.  Ten rounds of the  */
/* 4x32 S-box with the published multipliers and Weyl key increments.        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* golden ratio */
      k1 += 0xBB67AE85u; /* sqrt(3) - 1  */
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void orc_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  for (int64_t j = 0; j < n; ++j) orc_philox4x32_10(ctr + 4 * j, key + 2 * j, out + 4 * j);
}

/* Open-interval uniforms from Philox words.
 *   52-bit: k = (a << 20) | (b >> 12),  u = (k + 1/2) 2^-52
 *   23-bit: k = a >> 9,                 u = (k + 1/2) 2^-23
 * Both are exact in their precision and never reach 0 or 1. */
double orc_uniform52(uint32_t a, uint32_t b) {
  uint64_t k = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
  return ((double)k + 0.5) * 0x1p-52;
}

double orc_uniform23(uint32_t a) {
  uint32_t k = a >> 9;
  return ((double)k + 0.5) * 0x1p-23;
}

/* Uniforms (u1, u2, u3) of rejection trial m for link (site, mu) in heatbath
 * sweep number n.  key = (seed lo, seed hi), counter = (site, mu + 4 j, n lo,
 * n hi).  52-bit draws: trial m reads blocks j = 2m (u1 = words 0,1; u2 =
 * words 2,3) and 2m+1 (u3 = words 0,1).  23-bit draws: trials 2j and 2j+1
 * share block j; trial 2j takes words 0 and 1, trial 2j+1 words 2 and 3, as
 * u1 and u2, and u3 is the 23-bit uniform of u1's word shifted left by 23
 * (its nine low bits, which u1 does not use, so u3 > 1/2 exactly when bit 8
 * of that word is set). */
static void link_uniforms(const orc_params *p, uint32_t site, int mu, uint64_t n, int m, double u[3]) {
  uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
  uint32_t out0[4], out1[4];
  if (p->draws == 0) {
    uint32_t c0[4] = {site, (uint32_t)(mu + 4 * (2 * m)), (uint32_t)n, (uint32_t)(n >> 32)};
    uint32_t c1[4] = {site, (uint32_t)(mu + 4 * (2 * m + 1)), (uint32_t)n, (uint32_t)(n >> 32)};
    orc_philox4x32_10(c0, key, out0);
    orc_philox4x32_10(c1, key, out1);
    u[0] = orc_uniform52(out0[0], out0[1]);
    u[1] = orc_uniform52(out0[2], out0[3]);
    u[2] = orc_uniform52(out1[0], out1[1]);
  } else {
    uint32_t c0[4] = {site, (uint32_t)(mu + 4 * (m >> 1)), (uint32_t)n, (uint32_t)(n >> 32)};
    orc_philox4x32_10(c0, key, out0);
    const int w = 2 * (m & 1);
    u[0] = orc_uniform23(out0[w]);
    u[1] = orc_uniform23(out0[w + 1]);
    u[2] = orc_uniform23(out0[w] << 23);
  }
}

/* ------------------------------------------------------------------------ */
/* Von Mises sampler of Best & Fisher, "Efficient simulation of the von     */
/* Mises distribution", Applied Statistics 28 (1979) 152-157: draws psi on  */
/* (-pi, pi] with density exp(kappa cos psi) / (2 pi I0(kappa)).            */
/* ------------------------------------------------------------------------ */
#define ORC_KAPPA_TINY 1e-150 /* below this the law is uniform to 1e-150 */

/* Returns 0 and sets *psi, or -1 when the trial cap is reached. */
static int vonmises(const orc_params *p, double kappa, uint32_t site, int mu, uint64_t n, double *psi) {
  double u[3];
  if (kappa < ORC_KAPPA_TINY) {
    link_uniforms(p, site, mu, n, 0, u);
    *psi = ORC_PI * (2.0 * u[0] - 1.0);
    return 0;
  }
  /* tau = 1 + sqrt(1 + 4 kappa^2); rho = (tau - sqrt(2 tau)) / (2 kappa);
   * s = (1 + rho^2) / (2 rho).  tau - sqrt(2 tau) = tau (tau - 2) / (tau +
   * sqrt(2 tau)) and tau - 2 = 4 kappa^2 / (1 + sqrt(1 + 4 kappa^2)), which
   * keeps rho accurate when kappa is small. */
  double root = sqrt(1.0 + 4.0 * kappa * kappa);
  double tau = 1.0 + root;
  double tau_minus_2 = 4.0 * kappa * kappa / (1.0 + root);
  double rho = tau * tau_minus_2 / (tau + sqrt(2.0 * tau)) / (2.0 * kappa);
  double s = (1.0 + rho * rho) / (2.0 * rho);
  for (int m = 0; m < ORC_MAX_TRIALS; ++m) {
    link_uniforms(p, site, mu, n, m, u);
    double z = cos(ORC_PI * u[0]);
    double f = (1.0 + s * z) / (s + z);
    if (f > 1.0) f = 1.0;
    if (f < -1.0) f = -1.0;
    double c = kappa * (s - f);
    int accept = (c * (2.0 - c) - u[1] > 0.0) || (log(c / u[1]) + 1.0 - c >= 0.0);
    if (accept) {
      double a = acos(f);
      *psi = (u[2] > 0.5) ? a : -a;
      return 0;
    }
  }
  return -1;
}

/* Draw n samples of the von Mises law with the heatbath stream of site i,
 * direction 0, sweep 1 (i = 0 .. n-1).  Used by the sampler histogram test. */
int orc_vonmises_samples(const orc_params *p, double kappa, int64_t n, double *out) {
  int bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (vonmises(p, kappa, (uint32_t)i, 0, 1, &out[i]) != 0) bad = 1;
  }
  return bad ? ORC_EREJECT : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int L, Nt;
  int64_t V, Ns;
} geom;

static geom make_geom(const orc_params *p) {
  geom g;
  g.L = p->L;
  g.Nt = p->Nt;
  g.Ns = (int64_t)p->L * p->L * p->L;
  g.V = g.Ns * p->Nt;
  return g;
}

static void coords(const geom *g, int64_t i, int c[4]) {
  /* c[0] = t, c[1] = x, c[2] = y, c[3] = z */
  c[1] = (int)(i % g->L);
  i /= g->L;
  c[2] = (int)(i % g->L);
  i /= g->L;
  c[3] = (int)(i % g->L);
  i /= g->L;
  c[0] = (int)i;
}

static int64_t index_of(const geom *g, const int c[4]) {
  return (int64_t)c[1] + (int64_t)g->L * ((int64_t)c[2] + (int64_t)g->L * ((int64_t)c[3] + (int64_t)g->L * c[0]));
}

/* site i shifted by (d0, d1, d2, d3) along (t, x, y, z), periodic */
static int64_t shift(const geom *g, int64_t i, int d0, int d1, int d2, int d3) {
  int c[4];
  coords(g, i, c);
  int ext[4] = {g->Nt, g->L, g->L, g->L};
  int d[4] = {d0, d1, d2, d3};
  for (int a = 0; a < 4; ++a) {
    int v = (c[a] + d[a]) % ext[a];
    if (v < 0) v += ext[a];
    c[a] = v;
  }
  return index_of(g, c);
}

static int64_t step(const geom *g, int64_t i, int mu, int sign) {
  int d[4] = {0, 0, 0, 0};
  d[mu] = sign;
  return shift(g, i, d[0], d[1], d[2], d[3]);
}

static double wrap(double a) { return a - ORC_TWO_PI * floor((a + ORC_PI) / ORC_TWO_PI); }

/* ------------------------------------------------------------------------ */
/* Wilson action (Section II, eq. for S_g) and the staple sum               */
/* ------------------------------------------------------------------------ */

/* Sum of the six staples around U_mu(i): the local Boltzmann weight of
 * theta_mu(i) is exp(beta Re(e^{i theta_mu(i)} W)). */
void orc_staple(int L, int Nt, const double *th, int mu, int64_t i, double *wr, double *wi) {
  orc_params pp;
  memset(&pp, 0, sizeof pp);
  pp.L = L;
  pp.Nt = Nt;
  geom g = make_geom(&pp);
  const int64_t V = g.V;
  double re = 0.0, im = 0.0;
  int64_t ipmu = step(&g, i, mu, +1);
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    int64_t ipnu = step(&g, i, nu, +1);
    int64_t imnu = step(&g, i, nu, -1);
    int64_t ipmu_mnu = step(&g, ipmu, nu, -1);
    /* forward staple: U_nu(x+mu) U_mu(x+nu)^* U_nu(x)^* */
    double a = th[nu * V + ipmu] - th[mu * V + ipnu] - th[nu * V + i];
    /* backward staple: U_nu(x+mu-nu)^* U_mu(x-nu)^* U_nu(x-nu) */
    double b = -th[nu * V + ipmu_mnu] - th[mu * V + imnu] + th[nu * V + imnu];
    re += cos(a) + cos(b);
    im += sin(a) + sin(b);
  }
  *wr = re;
  *wi = im;
}

/* Plaquette angle theta_mu(x) + theta_nu(x+mu) - theta_mu(x+nu) - theta_nu(x) */
static double plaquette_angle(const geom *g, const double *th, int mu, int nu, int64_t i) {
  const int64_t V = g->V;
  return th[mu * V + i] + th[nu * V + step(g, i, mu, +1)] - th[mu * V + step(g, i, nu, +1)] - th[nu * V + i];
}

/* Mean over sites and the six planes of Re P_{mu nu} */
double orc_plaquette_mean(int L, int Nt, const double *th) {
  orc_params pp;
  memset(&pp, 0, sizeof pp);
  pp.L = L;
  pp.Nt = Nt;
  geom g = make_geom(&pp);
  double sum = 0.0;
  for (int64_t i = 0; i < g.V; ++i)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) sum += cos(plaquette_angle(&g, th, mu, nu, i));
  return sum / (6.0 * (double)g.V);
}

/* Total Wilson action S = beta sum_x sum_{mu<nu} Re(1 - P_{mu nu}(x)) */
double orc_action(int L, int Nt, double beta, const double *th) {
  orc_params pp;
  memset(&pp, 0, sizeof pp);
  pp.L = L;
  pp.Nt = Nt;
  geom g = make_geom(&pp);
  double sum = 0.0;
  for (int64_t i = 0; i < g.V; ++i)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) sum += 1.0 - cos(plaquette_angle(&g, th, mu, nu, i));
  return beta * sum;
}

/* Field components c = 0..5 -> plaquette planes:
 *   Ex, Ey, Ez = P_{01}, P_{02}, P_{03};  Bx, By, Bz = P_{23}, P_{31}, P_{12} */
static const int comp_mu[6] = {0, 0, 0, 2, 3, 1};
static const int comp_nu[6] = {1, 2, 3, 3, 1, 2};

/* Re and Im of P_c at every site: out[(2 c + k) V + i], k = 0 Re, 1 Im */
void orc_plaquette_field(int L, int Nt, const double *th, double *out) {
  orc_params pp;
  memset(&pp, 0, sizeof pp);
  pp.L = L;
  pp.Nt = Nt;
  geom g = make_geom(&pp);
  for (int c = 0; c < 6; ++c)
    for (int64_t i = 0; i < g.V; ++i) {
      double a = plaquette_angle(&g, th, comp_mu[c], comp_nu[c], i);
      out[(2 * c) * g.V + i] = cos(a);
      out[(2 * c + 1) * g.V + i] = sin(a);
    }
}

/* ------------------------------------------------------------------------ */
/* Configuration start and link updates                                     */
/* ------------------------------------------------------------------------ */

/* Hot start: theta = -pi + 2 pi u, u from block 0 of counter (i, mu, 0, 0). */
void orc_hot_start(const orc_params *p, double *th) {
  geom g = make_geom(p);
  uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
  for (int mu = 0; mu < 4; ++mu)
    for (int64_t i = 0; i < g.V; ++i) {
      uint32_t c[4] = {(uint32_t)i, (uint32_t)mu, 0u, 0u}, o[4];
      orc_philox4x32_10(c, key, o);
      th[mu * g.V + i] = -ORC_PI + ORC_TWO_PI * orc_uniform52(o[0], o[1]);
    }
}

static int parity_of(const geom *g, int64_t i) {
  int c[4];
  coords(g, i, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* Metropolis update of one link (Section II: the standard Metropolis
 * algorithm; the paper does not give its proposal, so it is a parameter): for
 * hit h = 0 .. metro_hits-1 with the uniforms (u1, u2) of trial h of the
 * heatbath stream, propose theta' = wrap(theta + w (2 u1 - 1)) and accept it
 * when u2 < exp(beta k [cos(theta' + alpha) - cos(theta + alpha)]), the ratio
 * of the link's weights exp(beta k cos(theta + alpha)) under the Wilson
 * action (always when the exponent is not negative). */
static double metropolis(const orc_params *p, double k, double alpha, uint32_t site, int mu, uint64_t n,
                         double theta) {
  for (int h = 0; h < p->metro_hits; ++h) {
    double u[3];
    link_uniforms(p, site, mu, n, h, u);
    double prop = wrap(theta + p->metro_width * (2.0 * u[0] - 1.0));
    double ds = p->beta * k * (cos(prop + alpha) - cos(theta + alpha));
    if (ds >= 0.0 || u[1] < exp(ds)) theta = prop;
  }
  return theta;
}

/* A spatial link on a time slice t = 0 (mod d) is frozen in slab mode d > 0. */
static int frozen(const geom *g, int64_t i, int mu, int d) {
  if (d <= 0 || mu == 0) return 0;
  int c[4];
  coords(g, i, c);
  return (c[0] % d) == 0;
}

/* One pass over the links U_mu(x) with parity(x) = par that are not frozen.
 * kind 0: heatbath theta <- wrap(psi - alpha), psi ~ vonMises(beta k);
 * kind 1: overrelaxation theta <- wrap(-2 alpha - theta) (k = 0: unchanged);
 * kind 2: Metropolis (metro_hits hits of half-width metro_width).
 * n is the update sweep number that keys the random stream. */
int orc_update_pass(const orc_params *p, double *th, int mu, int par, int d, uint64_t n, int kind) {
  geom g = make_geom(p);
  int bad = 0;
#ifdef _OPENMP
  int nthreads = p->threads > 0 ? p->threads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : bad)
#endif
  for (int64_t i = 0; i < g.V; ++i) {
    if (parity_of(&g, i) != par || frozen(&g, i, mu, d)) continue;
    double wr, wi;
    orc_staple(p->L, p->Nt, th, mu, i, &wr, &wi);
    double k = sqrt(wr * wr + wi * wi);
    double alpha = atan2(wi, wr);
    if (kind == 0) {
      double psi;
      if (vonmises(p, p->beta * k, (uint32_t)i, mu, n, &psi) != 0) {
        bad = 1;
        continue;
      }
      th[mu * g.V + i] = wrap(psi - alpha);
    } else if (kind == 2) {
      th[mu * g.V + i] = metropolis(p, k, alpha, (uint32_t)i, mu, n, th[mu * g.V + i]);
    } else {
      if (k == 0.0) continue;
      th[mu * g.V + i] = wrap(-2.0 * alpha - th[mu * g.V + i]);
    }
  }
  return bad ? ORC_EREJECT : ORC_OK;
}

/* Compound sweep (Section II: one update + n_or overrelaxations): update
 * sweep number ++(*counter) (heatbath, or Metropolis with update = 1), then
 * n_or overrelaxation sweeps.  Each sweep visits mu = 0, 1, 2, 3 and within
 * each direction the even sites before the odd ones (Section II.D: in-place
 * even/odd update). */
int orc_compound_sweep(const orc_params *p, double *th, int d, uint64_t *counter) {
  int status = ORC_OK;
  uint64_t n = ++(*counter);
  const int kind = p->update == 1 ? 2 : 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int par = 0; par < 2; ++par)
      if (orc_update_pass(p, th, mu, par, d, n, kind) != ORC_OK) status = ORC_EREJECT;
  for (int o = 0; o < p->n_or; ++o)
    for (int mu = 0; mu < 4; ++mu)
      for (int par = 0; par < 2; ++par) orc_update_pass(p, th, mu, par, d, n, 1);
  return status;
}

int orc_thermalize(const orc_params *p, double *th, uint64_t *counter, int n_sweeps) {
  int status = ORC_OK;
  for (int s = 0; s < n_sweeps; ++s)
    if (orc_compound_sweep(p, th, 0, counter) != ORC_OK) status = ORC_EREJECT;
  return status;
}

/* ------------------------------------------------------------------------ */
/* Observables: Polyakov loops, two-link operators and field insertions     */
/* ------------------------------------------------------------------------ */

/* P(x) = prod_t U_0(x, t) for every spatial site x (Section II.B). */
void orc_polyakov(int L, int Nt, const double *th, double *re, double *im) {
  orc_params pp;
  memset(&pp, 0, sizeof pp);
  pp.L = L;
  pp.Nt = Nt;
  geom g = make_geom(&pp);
  for (int64_t xs = 0; xs < g.Ns; ++xs) {
    double pr = 1.0, pi = 0.0;
    for (int t = 0; t < g.Nt; ++t) {
      double a = th[0 * g.V + xs + g.Ns * t];
      double cr = cos(a), ci = sin(a);
      double nr = pr * cr - pi * ci, ni = pr * ci + pi * cr;
      pr = nr;
      pi = ni;
    }
    re[xs] = pr;
    im[xs] = pi;
  }
}

/* Naive estimator (1/N_sigma) sum_x P(x)^* P(x + r xhat) on one configuration. */
static void naive_correlator(const geom *g, const double *th, int r, double *re, double *im) {
  double *pr = (double *)malloc(sizeof(double) * g->Ns);
  double *pi = (double *)malloc(sizeof(double) * g->Ns);
  orc_polyakov(g->L, g->Nt, th, pr, pi);
  double sr = 0.0, si = 0.0;
  for (int64_t xs = 0; xs < g->Ns; ++xs) {
    int64_t xr = shift(g, xs, 0, r, 0, 0);
    /* conj(P(x)) P(x+r) */
    sr += pr[xs] * pr[xr] + pi[xs] * pi[xr];
    si += pr[xs] * pi[xr] - pi[xs] * pr[xr];
  }
  *re = sr / (double)g->Ns;
  *im = si / (double)g->Ns;
  free(pr);
  free(pi);
}

void orc_naive_correlator(int L, int Nt, const double *th, int r, double *re, double *im) {
  orc_params pp;
  memset(&pp, 0, sizeof pp);
  pp.L = L;
  pp.Nt = Nt;
  geom g = make_geom(&pp);
  naive_correlator(&g, th, r, re, im);
}

/* Two-link operator T(x, t, r) = U_0(x, t)^* U_0(x + r xhat, t) (Section
 * II.C), multiplied over the d time slices t0 .. t0+d-1 of one slab. */
static void slab_two_link(const geom *g, const double *th, int64_t xs, int t0, int d, int r, double *re,
                          double *im) {
  double pr = 1.0, pi = 0.0;
  int64_t xr = shift(g, xs, 0, r, 0, 0);
  for (int t = t0; t < t0 + d; ++t) {
    double a = th[0 * g->V + xs + g->Ns * t];
    double b = th[0 * g->V + xr + g->Ns * t];
    /* U_0(x,t)^* U_0(x+r,t) */
    double tr = cos(a) * cos(b) + sin(a) * sin(b);
    double ti = cos(a) * sin(b) - sin(a) * cos(b);
    double nr = pr * tr - pi * ti, ni = pr * ti + pi * tr;
    pr = nr;
    pi = ni;
  }
  *re = pr;
  *im = pi;
}

/* Modified Bessel functions of the first kind from their power series,
 * I_n(x) = sum_k (x/2)^(2k+n) / (k! (k+n)!), summed until the terms stop
 * changing the sum (x >= 0). */
static double bessel_i(int n, double x) {
  const double h = 0.5 * x, h2 = h * h;
  double term = 1.0;
  for (int j = 1; j <= n; ++j) term *= h / j; /* (x/2)^n / n! */
  double sum = term;
  for (int k = 1; k < 100000; ++k) {
    term *= h2 / ((double)k * (double)(k + n));
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

double orc_bessel_i0(double x) { return bessel_i(0, x); }
double orc_bessel_i1(double x) { return bessel_i(1, x); }

/* Analytic multihit (Section II.C: the innermost average of a temporal link
 * with every other link fixed): the conditional mean of U_0(x, t) under the
 * weight exp(beta k cos(theta + alpha)) of its staple sum k e^{i alpha},
 *   <U_0> = e^{-i alpha} I1(beta k) / I0(beta k). */
static void multihit_link(const orc_params *p, const double *th, int64_t i, double *re, double *im) {
  double wr, wi;
  orc_staple(p->L, p->Nt, th, 0, i, &wr, &wi);
  const double k = sqrt(wr * wr + wi * wi);
  const double alpha = atan2(wi, wr);
  const double ratio = k > 0.0 ? orc_bessel_i1(p->beta * k) / orc_bessel_i0(p->beta * k) : 0.0;
  *re = ratio * cos(alpha);
  *im = -ratio * sin(alpha);
}

void orc_multihit_link(const orc_params *p, const double *th, int64_t i, double out[2]) {
  multihit_link(p, th, i, &out[0], &out[1]);
}

/* Slab product of the multihit temporal links, prod_{t in slab} <U_0(x, t)>. */
static void slab_multihit(const orc_params *p, const geom *g, const double *th, int64_t xs, int t0, int d,
                          double *re, double *im) {
  double pr = 1.0, pi = 0.0;
  for (int t = t0; t < t0 + d; ++t) {
    double ur, ui;
    multihit_link(p, th, xs + g->Ns * t, &ur, &ui);
    const double nr = pr * ur - pi * ui, ni = pr * ui + pi * ur;
    pr = nr;
    pi = ni;
  }
  *re = pr;
  *im = pi;
}

/* ------------------------------------------------------------------------ */
/* Multilevel measurement (Algorithm 1; Section II.C)                        */
/* ------------------------------------------------------------------------ */

/* Length of one measurement record:
 *   P      [nr][2]                 (Re, Im) of (1/N_s) sum_x prod_s [T]_s
 *   Pf     [nrf][2]                the same at the field separations rf
 *   W      [nrf][nprobe][6][2][2]  component c, insertion k (Re P / Im P),
 *                                  (Re, Im) of (1/(N_s N_t)) sum_x sum_s
 *                                  [TO]_s prod_{s' != s} [T]_{s'}
 *   vac    [6][2]                  mean of Re P_c, Im P_c over sites and the
 *                                  sub-update configurations of the measurement
 *   naive  [nr][2]                 naive P+P on the measurement's first config
 *   plaq   [1]                     mean plaquette of that configuration       */
int64_t orc_record_len(const orc_params *p) {
  return (int64_t)p->nr * 2 + (int64_t)p->nrf * 2 + (int64_t)p->nrf * p->nprobe * 24 + 12 + (int64_t)p->nr * 2 + 1;
}

typedef struct {
  double re, im;
} cplx;

static cplx cmul(cplx a, cplx b) {
  cplx c = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return c;
}

static int validate(const orc_params *p) {
  if (p->L < 2 || p->Nt < 2 || (p->L & 1) || (p->Nt & 1)) return ORC_EINVAL;
  if (p->beta < 0.0 || p->n_or < 0 || p->draws < 0 || p->draws > 1) return ORC_EINVAL;
  if (p->update < 0 || p->update > 1 || p->multihit < 0 || p->multihit > 1) return ORC_EINVAL;
  if (p->multihit && p->beta > 100.0) return ORC_EINVAL; /* I0(beta k) stays finite for k <= 6 */
  if (p->update == 1 && (p->metro_hits < 1 || p->metro_hits > ORC_MAX_TRIALS || !(p->metro_width > 0.0) ||
                         p->metro_width > ORC_PI))
    return ORC_EINVAL;
  if (p->slab < 1 || p->Nt % p->slab != 0 || p->n_sub < 1 || p->k_between < 0) return ORC_EINVAL;
  if (p->outer_slab != 0) {
    if (p->outer_slab % p->slab != 0 || p->Nt % p->outer_slab != 0 || p->outer_slab == p->slab) return ORC_EINVAL;
    if (p->n_sub_outer < 1) return ORC_EINVAL;
  }
  for (int a = 0; a < p->nr; ++a)
    if (p->r[a] < 1 || p->r[a] >= p->L) return ORC_EINVAL;
  for (int a = 0; a < p->nrf; ++a)
    if (p->rf[a] < 1 || p->rf[a] >= p->L) return ORC_EINVAL;
  for (int a = 0; a < p->nprobe; ++a)
    if (abs(p->probe_dy[a]) >= p->L || abs(p->probe_dz[a]) >= p->L) return ORC_EINVAL;
  if (p->comp_mask >= 64u) return ORC_EINVAL;
  return ORC_OK;
}

int orc_validate(const orc_params *p) { return validate(p); }

/* Per-slab sub-averages of one level: [T](x, r) for the separations of both
 * lists and [TO](x, rf, probe, c, k), summed over the sub-updates. */
typedef struct {
  int nslab;
  cplx *t_pr;  /* [nslab][nr][Ns]                 */
  cplx *t_fr;  /* [nslab][nrf][Ns]                */
  cplx *to;    /* [nslab][nrf][nprobe][6][2][Ns]  */
} slab_sums;

static int alloc_sums(const orc_params *p, const geom *g, int nslab, slab_sums *s) {
  s->nslab = nslab;
  size_t ns = (size_t)g->Ns;
  s->t_pr = (cplx *)calloc((size_t)nslab * p->nr * ns + 1, sizeof(cplx));
  s->t_fr = (cplx *)calloc((size_t)nslab * p->nrf * ns + 1, sizeof(cplx));
  s->to = (cplx *)calloc((size_t)nslab * p->nrf * p->nprobe * 12 * ns + 1, sizeof(cplx));
  return (s->t_pr && s->t_fr && s->to) ? ORC_OK : ORC_ENOMEM;
}

static void zero_sums(const orc_params *p, const geom *g, slab_sums *s) {
  size_t ns = (size_t)g->Ns;
  memset(s->t_pr, 0, sizeof(cplx) * s->nslab * p->nr * ns);
  memset(s->t_fr, 0, sizeof(cplx) * s->nslab * p->nrf * ns);
  memset(s->to, 0, sizeof(cplx) * s->nslab * p->nrf * p->nprobe * 12 * ns);
}

static void free_sums(slab_sums *s) {
  free(s->t_pr);
  free(s->t_fr);
  free(s->to);
}

#define T_PR(S, sl, a, x) ((S)->t_pr[((size_t)(sl) * p->nr + (a)) * g->Ns + (x)])
#define T_FR(S, sl, a, x) ((S)->t_fr[((size_t)(sl) * p->nrf + (a)) * g->Ns + (x)])
#define T_O(S, sl, a, b, c, k, x) \
  ((S)->to[(((((size_t)(sl) * p->nrf + (a)) * p->nprobe + (b)) * 6 + (c)) * 2 + (k)) * g->Ns + (x)])

/* Accumulate T^(d) and TO^(d) of the current configuration into the inner
 * sums (Section II.C, eqs. for T^(2) and TO^(2), with thickness d), and the
 * plaquette vacuum sums. */
static void accumulate_inner(const orc_params *p, const geom *g, const double *th, slab_sums *S, double *pf,
                             double vac[12]) {
  const int d = p->slab;
  orc_plaquette_field(g->L, g->Nt, th, pf);
  for (int c = 0; c < 6; ++c) {
    if (!(p->comp_mask & (1u << c))) continue;
    for (int k = 0; k < 2; ++k) {
      double sum = 0.0;
      for (int64_t i = 0; i < g->V; ++i) sum += pf[(2 * c + k) * g->V + i];
      vac[2 * c + k] += sum / (double)g->V;
    }
  }
#ifdef _OPENMP
  int nthreads = p->threads > 0 ? p->threads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int64_t xs = 0; xs < g->Ns; ++xs) {
    for (int sl = 0; sl < S->nslab; ++sl) {
      int t0 = sl * d;
      for (int a = 0; a < p->nr; ++a) {
        cplx t;
        if (p->multihit && p->r[a] >= 2 && p->L - p->r[a] >= 2) {
          /* lines two or more sites apart (both ways round the torus) share
           * no plaquette: each link is replaced by its multihit mean,
           * conj(prod <U_0>(x)) prod <U_0>(x + r) */
          double ar, ai, br, bi;
          slab_multihit(p, g, th, xs, t0, d, &ar, &ai);
          slab_multihit(p, g, th, shift(g, xs, 0, p->r[a], 0, 0), t0, d, &br, &bi);
          t.re = ar * br + ai * bi;
          t.im = ar * bi - ai * br;
        } else {
          slab_two_link(g, th, xs, t0, d, p->r[a], &t.re, &t.im);
        }
        T_PR(S, sl, a, xs).re += t.re;
        T_PR(S, sl, a, xs).im += t.im;
      }
      for (int a = 0; a < p->nrf; ++a) {
        cplx t;
        slab_two_link(g, th, xs, t0, d, p->rf[a], &t.re, &t.im);
        T_FR(S, sl, a, xs).re += t.re;
        T_FR(S, sl, a, xs).im += t.im;
        for (int b = 0; b < p->nprobe; ++b) {
          /* probe anchor x0 = x + floor(rf/2) xhat + (0, dy, dz) */
          int64_t x0 = shift(g, xs, 0, p->rf[a] / 2, p->probe_dy[b], p->probe_dz[b]);
          for (int c = 0; c < 6; ++c) {
            if (!(p->comp_mask & (1u << c))) continue;
            for (int k = 0; k < 2; ++k) {
              double o = 0.0;
              for (int t = t0; t < t0 + d; ++t) o += pf[(2 * c + k) * g->V + x0 + g->Ns * t];
              T_O(S, sl, a, b, c, k, xs).re += t.re * o;
              T_O(S, sl, a, b, c, k, xs).im += t.im * o;
            }
          }
        }
      }
    }
  }
}

/* Level combination (Algorithm 1, "Calculate [T2][T2]"; Section II.C eqs.
 * for T^(4) and TO^(4)): for each outer slab, whose inner slabs j = q S ..
 * q S + q - 1 carry the inner averages [T]_j = inner_sum / n2,
 *   outer T  += prod_j [T]_j
 *   outer TO += sum_j [TO]_j prod_{j' != j} [T]_{j'}                     */
static void combine_levels(const orc_params *p, const geom *g, const slab_sums *in, slab_sums *out) {
  const int q = p->outer_slab / p->slab;
  const double inv = 1.0 / (double)p->n_sub;
  for (int so = 0; so < out->nslab; ++so)
    for (int64_t xs = 0; xs < g->Ns; ++xs) {
      for (int a = 0; a < p->nr; ++a) {
        cplx prod = {1.0, 0.0};
        for (int j = 0; j < q; ++j) {
          cplx t = T_PR(in, q * so + j, a, xs);
          t.re *= inv;
          t.im *= inv;
          prod = cmul(prod, t);
        }
        T_PR(out, so, a, xs).re += prod.re;
        T_PR(out, so, a, xs).im += prod.im;
      }
      for (int a = 0; a < p->nrf; ++a) {
        cplx prod = {1.0, 0.0};
        for (int j = 0; j < q; ++j) {
          cplx t = T_FR(in, q * so + j, a, xs);
          t.re *= inv;
          t.im *= inv;
          prod = cmul(prod, t);
        }
        T_FR(out, so, a, xs).re += prod.re;
        T_FR(out, so, a, xs).im += prod.im;
        for (int b = 0; b < p->nprobe; ++b)
          for (int c = 0; c < 6; ++c) {
            if (!(p->comp_mask & (1u << c))) continue;
            for (int k = 0; k < 2; ++k) {
              cplx sum = {0.0, 0.0};
              for (int j = 0; j < q; ++j) {
                cplx term = T_O(in, q * so + j, a, b, c, k, xs);
                term.re *= inv;
                term.im *= inv;
                for (int jj = 0; jj < q; ++jj) {
                  if (jj == j) continue;
                  cplx t = T_FR(in, q * so + jj, a, xs);
                  t.re *= inv;
                  t.im *= inv;
                  term = cmul(term, t);
                }
                sum.re += term.re;
                sum.im += term.im;
              }
              T_O(out, so, a, b, c, k, xs).re += sum.re;
              T_O(out, so, a, b, c, k, xs).im += sum.im;
            }
          }
      }
    }
}

/* Cross-slab products (Section II.C, eqs. for <P+P> and <P+P O>): with the
 * top-level averages [T]_s = sum / n,
 *   P(r)          = (1/N_s) sum_x prod_s [T]_s(x)
 *   W(rf, b, c, k) = (1/(N_s N_t)) sum_x sum_s [TO]_s(x) prod_{s' != s} [T]_{s'}(x) */
static void cross_slab(const orc_params *p, const geom *g, const slab_sums *S, double n, double *rec) {
  const double inv = 1.0 / n;
  for (int a = 0; a < p->nr; ++a) {
    double sr = 0.0, si = 0.0;
    for (int64_t xs = 0; xs < g->Ns; ++xs) {
      cplx prod = {1.0, 0.0};
      for (int sl = 0; sl < S->nslab; ++sl) {
        cplx t = T_PR(S, sl, a, xs);
        t.re *= inv;
        t.im *= inv;
        prod = cmul(prod, t);
      }
      sr += prod.re;
      si += prod.im;
    }
    rec[2 * a] = sr / (double)g->Ns;
    rec[2 * a + 1] = si / (double)g->Ns;
  }
  double *pf = rec + 2 * p->nr;
  for (int a = 0; a < p->nrf; ++a) {
    double sr = 0.0, si = 0.0;
    for (int64_t xs = 0; xs < g->Ns; ++xs) {
      cplx prod = {1.0, 0.0};
      for (int sl = 0; sl < S->nslab; ++sl) {
        cplx t = T_FR(S, sl, a, xs);
        t.re *= inv;
        t.im *= inv;
        prod = cmul(prod, t);
      }
      sr += prod.re;
      si += prod.im;
    }
    pf[2 * a] = sr / (double)g->Ns;
    pf[2 * a + 1] = si / (double)g->Ns;
  }
  double *w = pf + 2 * p->nrf;
  for (int a = 0; a < p->nrf; ++a)
    for (int b = 0; b < p->nprobe; ++b)
      for (int c = 0; c < 6; ++c)
        for (int k = 0; k < 2; ++k) {
          double sr = 0.0, si = 0.0;
          if (p->comp_mask & (1u << c)) {
            for (int64_t xs = 0; xs < g->Ns; ++xs)
              for (int sl = 0; sl < S->nslab; ++sl) {
                cplx term = T_O(S, sl, a, b, c, k, xs);
                term.re *= inv;
                term.im *= inv;
                for (int s2 = 0; s2 < S->nslab; ++s2) {
                  if (s2 == sl) continue;
                  cplx t = T_FR(S, s2, a, xs);
                  t.re *= inv;
                  t.im *= inv;
                  term = cmul(term, t);
                }
                sr += term.re;
                si += term.im;
              }
          }
          size_t o = ((((size_t)a * p->nprobe + b) * 6 + c) * 2 + k) * 2;
          w[o] = sr / ((double)g->Ns * g->Nt);
          w[o + 1] = si / ((double)g->Ns * g->Nt);
        }
}

/* ------------------------------------------------------------------------ */
/* One measurement from configurations the caller supplies (Algorithm 1's     */
/* accumulation and products without its sweeps).  orc_measure below drives  */
/* the same functions with its own sweeps; tests feed them configurations     */
/* taken from elsewhere (another chain, or built by hand).                    */
/* ------------------------------------------------------------------------ */
typedef struct orc_acc orc_acc;
struct orc_acc {
  orc_params p;
  geom g;
  int two_level;
  slab_sums inner, outer;
  double *pf;    /* plaquette field of the configuration being accumulated */
  double *rec;   /* the record being formed                                */
  double vac[12];
  int n_cfg;     /* sub-update configurations accumulated                  */
  int n_inner;   /* of them since the last level combination               */
  int n_outer;   /* level combinations done                                */
};

static double *naive_block(const orc_params *p, double *rec) {
  return rec + 2 * p->nr + 2 * p->nrf + (size_t)p->nrf * p->nprobe * 24 + 12;
}

void orc_acc_free(orc_acc *a) {
  if (!a) return;
  free(a->pf);
  free(a->rec);
  free_sums(&a->inner);
  if (a->two_level) free_sums(&a->outer);
  free(a);
}

/* NULL when *p is invalid or memory runs out.  The lists of *p must outlive
 * the accumulator. */
orc_acc *orc_acc_create(const orc_params *p) {
  if (validate(p) != ORC_OK) return NULL;
  orc_acc *a = (orc_acc *)calloc(1, sizeof(orc_acc));
  if (!a) return NULL;
  a->p = *p;
  a->g = make_geom(p);
  a->two_level = p->outer_slab != 0;
  a->pf = (double *)malloc(sizeof(double) * 12 * a->g.V);
  a->rec = (double *)calloc((size_t)orc_record_len(p), sizeof(double));
  int ok = a->pf && a->rec && alloc_sums(p, &a->g, p->Nt / p->slab, &a->inner) == ORC_OK;
  if (ok && a->two_level) ok = alloc_sums(p, &a->g, p->Nt / p->outer_slab, &a->outer) == ORC_OK;
  if (!ok) {
    orc_acc_free(a);
    return NULL;
  }
  return a;
}

/* Start a measurement: clear the sums; the naive estimator and the plaquette
 * come from th_first, the configuration before the first sub-update. */
int orc_acc_begin(orc_acc *a, const double *th_first) {
  const orc_params *p = &a->p;
  memset(a->rec, 0, sizeof(double) * (size_t)orc_record_len(p));
  memset(a->vac, 0, sizeof a->vac);
  zero_sums(p, &a->g, &a->inner);
  if (a->two_level) zero_sums(p, &a->g, &a->outer);
  a->n_cfg = a->n_inner = a->n_outer = 0;
  double *naive = naive_block(p, a->rec);
  for (int r = 0; r < p->nr; ++r) naive_correlator(&a->g, th_first, p->r[r], &naive[2 * r], &naive[2 * r + 1]);
  naive[2 * p->nr] = orc_plaquette_mean(p->L, p->Nt, th_first);
  return ORC_OK;
}

/* Accumulate T^(d) and TO^(d) of one (inner) sub-update configuration. */
int orc_acc_add(orc_acc *a, const double *th) {
  accumulate_inner(&a->p, &a->g, th, &a->inner, a->pf, a->vac);
  ++a->n_cfg;
  ++a->n_inner;
  return ORC_OK;
}

/* Two levels: fold the inner averages of the n_sub configurations added since
 * the last call into the outer sums (Algorithm 1's level combination) and
 * clear the inner sums. */
int orc_acc_end_outer(orc_acc *a) {
  if (!a->two_level || a->n_inner != a->p.n_sub) return ORC_EINVAL;
  combine_levels(&a->p, &a->g, &a->inner, &a->outer);
  zero_sums(&a->p, &a->g, &a->inner);
  a->n_inner = 0;
  ++a->n_outer;
  return ORC_OK;
}

/* Cross-slab products of the top-level averages (the P, Pf and W blocks),
 * the vacuum means, and the naive block of orc_acc_begin into rec
 * (orc_record_len doubles).  One level needs exactly n_sub added
 * configurations, two levels exactly n_sub_outer combinations. */
int orc_acc_finish(orc_acc *a, double *rec) {
  const orc_params *p = &a->p;
  if (a->two_level ? (a->n_outer != p->n_sub_outer || a->n_inner != 0) : a->n_inner != p->n_sub) return ORC_EINVAL;
  if (a->two_level)
    cross_slab(p, &a->g, &a->outer, (double)p->n_sub_outer, a->rec);
  else
    cross_slab(p, &a->g, &a->inner, (double)p->n_sub, a->rec);
  double *v = a->rec + 2 * p->nr + 2 * p->nrf + (size_t)p->nrf * p->nprobe * 24;
  for (int c = 0; c < 12; ++c) v[c] = a->vac[c] / (double)a->n_cfg;
  memcpy(rec, a->rec, sizeof(double) * (size_t)orc_record_len(p));
  return ORC_OK;
}

/* n_meas multilevel measurements (Algorithm 1).  Each one: k0 full compound
 * sweeps; then either
 *   single level: n2 slab sub-updates (spatial links frozen on t = 0 mod d),
 *                 each followed by the accumulation of T^(d) and TO^(d);
 *   two level:    n4 outer iterations, each one compound sweep with the outer
 *                 mask (t = 0 mod D) followed by the single-level inner loop
 *                 and the level combination;
 * and finally the cross-slab products.  rec receives n_meas records of
 * orc_record_len(p) doubles.  *counter is the heatbath sweep number. */
int orc_measure(const orc_params *p, double *th, uint64_t *counter, int n_meas, double *rec) {
  int status = validate(p);
  if (status != ORC_OK) return status;
  orc_acc *a = orc_acc_create(p);
  if (!a) return ORC_ENOMEM;
  const int64_t len = orc_record_len(p);
  for (int m = 0; m < n_meas; ++m) {
    for (int s = 0; s < p->k_between; ++s)
      if (orc_compound_sweep(p, th, 0, counter) != ORC_OK) status = ORC_EREJECT;
    orc_acc_begin(a, th);
    const int n_outer = a->two_level ? p->n_sub_outer : 1;
    for (int o = 0; o < n_outer; ++o) {
      if (a->two_level && orc_compound_sweep(p, th, p->outer_slab, counter) != ORC_OK) status = ORC_EREJECT;
      for (int j = 0; j < p->n_sub; ++j) {
        if (orc_compound_sweep(p, th, p->slab, counter) != ORC_OK) status = ORC_EREJECT;
        orc_acc_add(a, th);
      }
      if (a->two_level) orc_acc_end_outer(a);
    }
    orc_acc_finish(a, rec + (size_t)m * len);
  }
  orc_acc_free(a);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Connected field profile from n_meas records (Section II.C, the connected */
/* expectation value of the field and the relations between the plaquette  */
/* and the field): with sums over the measurements,                          */
/*   <O>_{P+P} = (sum_m W_m) / (sum_m Re Pf_m) - (1/n) sum_m vac_m,          */
/*   F   = sqrt(beta) <Im P_c>_{P+P}   (k = 1 insertion),                    */
/*   F^2 = -2 beta <Re P_c>_{P+P}      (k = 0 insertion; the constant 1 of   */
/*                                      2 beta (1 - Re P) cancels between    */
/*                                      the two terms)                       */
/* from the real parts of W (the imaginary parts average to zero).  Errors  */
/* by the delete-one jackknife over measurements (Section III): the         */
/* estimate recomputed without measurement m, and                           */
/* err^2 = (n-1)/n sum_m (est_m - mean_m est_m)^2.                           */
/* out[nrf][nprobe][6][4] = (F, F^2, err F, err F^2); unselected components */
/* and n_meas < 2 give zero errors.                                          */
/* ------------------------------------------------------------------------ */
static void connected_of(const orc_params *p, const double *recs, int n_meas, int skip, int f, int b, int c,
                         double *F, double *F2) {
  const int64_t len = orc_record_len(p);
  const size_t off_pf = 2 * (size_t)p->nr;
  const size_t off_w = off_pf + 2 * (size_t)p->nrf;
  const size_t off_vac = off_w + (size_t)p->nrf * p->nprobe * 24;
  double pf = 0.0, w0 = 0.0, w1 = 0.0, v0 = 0.0, v1 = 0.0;
  int n = 0;
  for (int m = 0; m < n_meas; ++m) {
    if (m == skip) continue;
    const double *r = recs + (size_t)m * len;
    pf += r[off_pf + 2 * f];
    const size_t wo = off_w + ((((size_t)f * p->nprobe + b) * 6 + c) * 2) * 2;
    w0 += r[wo];     /* Re W of the Re P_c insertion */
    w1 += r[wo + 2]; /* Re W of the Im P_c insertion */
    v0 += r[off_vac + 2 * c];
    v1 += r[off_vac + 2 * c + 1];
    ++n;
  }
  *F = sqrt(p->beta) * (w1 / pf - v1 / n);
  *F2 = -2.0 * p->beta * (w0 / pf - v0 / n);
}

int orc_connected(const orc_params *p, const double *recs, int n_meas, double *out) {
  if (validate(p) != ORC_OK || n_meas < 1) return ORC_EINVAL;
  for (int f = 0; f < p->nrf; ++f)
    for (int b = 0; b < p->nprobe; ++b)
      for (int c = 0; c < 6; ++c) {
        double *o = out + ((((size_t)f * p->nprobe + b) * 6 + c) * 4);
        o[0] = o[1] = o[2] = o[3] = 0.0;
        if (!(p->comp_mask & (1u << c))) continue;
        connected_of(p, recs, n_meas, -1, f, b, c, &o[0], &o[1]);
        if (n_meas < 2) continue;
        double sF = 0.0, sF2 = 0.0;
        for (int m = 0; m < n_meas; ++m) {
          double F, F2;
          connected_of(p, recs, n_meas, m, f, b, c, &F, &F2);
          sF += F;
          sF2 += F2;
        }
        const double mF = sF / n_meas, mF2 = sF2 / n_meas;
        double eF = 0.0, eF2 = 0.0;
        for (int m = 0; m < n_meas; ++m) {
          double F, F2;
          connected_of(p, recs, n_meas, m, f, b, c, &F, &F2);
          eF += (F - mF) * (F - mF);
          eF2 += (F2 - mF2) * (F2 - mF2);
        }
        o[2] = sqrt((n_meas - 1.0) / n_meas * eF);
        o[3] = sqrt((n_meas - 1.0) / n_meas * eF2);
      }
  return ORC_OK;
}
