/*
 * Seeded synthetic inputs for the 2d U(1) Wilson-Dirac multigrid solver.
 *
 * This file holds NO arithmetic of the multigrid method itself. It only makes
 * the inputs that both the FP64 oracle and the CUDA library consume:
 *   - Philox4x32-10 counter-based random numbers (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the
 *     published round function: two 32x32->64 multiplies per round with the
 *     multipliers 0xD2511F53 / 0xCD9E8D57, and a Weyl key schedule with
 *     increments 0x9E3779B9 / 0xBB67AE85.
 *   - Complex Gaussian fields via the Box-Muller transform.
 *   - Quenched U(1) gauge links from a Metropolis Markov chain with the
 *     Wilson plaquette action S = beta * sum_p Re U_p (the paper's gauge
 *     ensembles: 2d, periodic, beta = 6 and 10), weight exp(+S).
 *   - Random U(1) gauge transformations (for covariance tests).
 *
 * Every routine is deterministic for a given seed and independent of the
 * number of OpenMP threads: the Metropolis sweep is split into four
 * sub-sweeps whose links share no plaquette, and every random number is
 * addressed by a counter, never drawn from a sequential stream.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off (no FMA contraction,
 * so x86_64 and aarch64 hosts produce the same bits up to libm rounding).
 *
 * Layouts (shared with the library's boundary):
 *   site index x = x0 + L0 * x1 (x0 fastest)
 *   link angle theta[x*2 + mu]   (U_x^mu = exp(i theta), mu = 0, 1)
 *   complex fields interleaved (re, im).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: out = F(ctr; key). */
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(PHILOX_M0, c0, &hi0, &lo0);
    mulhilo32(PHILOX_M1, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two 53-bit uniforms from one Philox block: u_a in (0,1], u_b in [0,1). */
static inline void two_uniforms(const uint32_t w[4], double *ua, double *ub) {
  uint64_t a = (((uint64_t)w[1] << 32) | w[0]) >> 11;
  uint64_t b = (((uint64_t)w[3] << 32) | w[2]) >> 11;
  const double s = 1.0 / 9007199254740992.0; /* 2^-53 */
  *ua = (double)(a + 1) * s;
  *ub = (double)b * s;
}

static inline void seed_key(uint64_t seed, uint32_t key[2]) {
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32);
}

/*
 * n complex Gaussians z_i = sqrt(-2 ln u1) * exp(2 pi i u2) with counter
 * (i_lo, i_hi, tag_lo, tag_hi) under key = seed. Re and Im are independent
 * N(0,1). Returns the field interleaved in out[2n].
 */
void gen_gaussian_complex(int64_t n, uint64_t seed, uint64_t tag, double *out) {
  uint32_t key[2];
  seed_key(seed, key);
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)tag, (uint32_t)(tag >> 32)};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    double u1, u2;
    two_uniforms(w, &u1, &u2);
    double rad = sqrt(-2.0 * log(u1));
    out[2 * i] = rad * cos(two_pi * u2);
    out[2 * i + 1] = rad * sin(two_pi * u2);
  }
}

/* n uniforms in [0,1) (counter (i_lo, i_hi, tag_lo, tag_hi)), for tests. */
void gen_uniform(int64_t n, uint64_t seed, uint64_t tag, double *out) {
  uint32_t key[2];
  seed_key(seed, key);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)tag, (uint32_t)(tag >> 32)};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    double ua, ub;
    two_uniforms(w, &ua, &ub);
    out[i] = ub;
  }
}

static inline int64_t site_of(int x0, int x1, int L0) { return (int64_t)x0 + (int64_t)L0 * x1; }

/*
 * Quenched U(1) Metropolis on an L0 x L1 periodic lattice (L0, L1 even).
 * theta[2*x + mu] is the link angle; on entry it holds the start (a cold
 * start is theta = 0). Each sweep visits every link `hits` times with
 * proposals theta' = theta + delta, delta uniform in [-step, step], accepted
 * with probability min(1, exp(beta * (Re U_p' - Re U_p) summed over the two
 * plaquettes that contain the link)).
 *
 * The four sub-sweeps are (mu=0, x1 even), (mu=0, x1 odd), (mu=1, x0 even),
 * (mu=1, x0 odd); links inside one sub-sweep share no plaquette, so they are
 * updated in parallel with a thread-count-independent result.
 * Random numbers: key = seed, counter = (x, sweep, mu + 2*hit, 0x4D45) with
 * u_a -> accept test, u_b -> delta.
 */
void metropolis_u1_2d(int L0, int L1, double beta, int sweeps, int hits, double step, uint64_t seed,
                      double *theta, int64_t *accepted_out) {
  uint32_t key[2];
  seed_key(seed, key);
  int64_t accepted = 0;
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int sub = 0; sub < 4; ++sub) {
      const int mu = sub >> 1, parity = sub & 1;
      /* links of direction mu whose coordinate in the other direction has this parity */
      const int n_other = (mu == 0) ? L1 / 2 : L0 / 2;
      const int n_along = (mu == 0) ? L0 : L1;
      const int64_t nwork = (int64_t)n_other * n_along;
#pragma omp parallel for schedule(static) reduction(+ : accepted)
      for (int64_t w = 0; w < nwork; ++w) {
        int along = (int)(w % n_along), other = 2 * (int)(w / n_along) + parity;
        int x0 = (mu == 0) ? along : other, x1 = (mu == 0) ? other : along;
        int x0p = (x0 + 1) % L0, x0m = (x0 + L0 - 1) % L0;
        int x1p = (x1 + 1) % L1, x1m = (x1 + L1 - 1) % L1;
        int64_t x = site_of(x0, x1, L0);
        /* plaquette angle theta_p(y) = t0(y) + t1(y+0) - t0(y+1) - t1(y).
           link (x,mu=0): +t0(x) in p(x), -t0(x) in p(x-1)
           link (x,mu=1): -t1(x) in p(x), +t1(x) in p(x-0)
           The plaquette where the link enters with + sign gives cos(t + a);
           the one where it enters with - sign gives cos(b - t) = cos(t - b). */
        double a, b;
        if (mu == 0) {
          a = theta[2 * site_of(x0p, x1, L0) + 1] - theta[2 * site_of(x0, x1p, L0) + 0] - theta[2 * x + 1];
          int64_t y = site_of(x0, x1m, L0); /* p(x - 1hat) */
          b = theta[2 * y + 0] + theta[2 * site_of(x0p, x1m, L0) + 1] - theta[2 * y + 1];
        } else {
          int64_t y = site_of(x0m, x1, L0); /* p(x - 0hat) */
          a = theta[2 * y + 0] - theta[2 * site_of(x0m, x1p, L0) + 0] - theta[2 * y + 1];
          b = theta[2 * x + 0] + theta[2 * site_of(x0p, x1, L0) + 1] - theta[2 * site_of(x0, x1p, L0) + 0];
        }
        /* staple sum: local action = beta * Re(e^{i t} * S), S = e^{i a} + e^{-i b} */
        const double Sr = cos(a) + cos(b), Si = sin(a) - sin(b);
        double t = theta[2 * x + mu];
        double local = cos(t) * Sr - sin(t) * Si;
        for (int h = 0; h < hits; ++h) {
          uint32_t ctr[4] = {(uint32_t)x, (uint32_t)sweep, (uint32_t)(mu + 2 * h), 0x4D45u};
          uint32_t rw[4];
          philox4x32_10(ctr, key, rw);
          double ua, ub;
          two_uniforms(rw, &ua, &ub);
          double tn = t + step * (2.0 * ub - 1.0);
          double local_n = cos(tn) * Sr - sin(tn) * Si;
          double dS = beta * (local_n - local);
          if (dS >= 0.0 || ua <= exp(dS)) {
            t = tn;
            local = local_n;
            ++accepted;
          }
        }
        /* keep the angle in (-pi, pi] */
        t = remainder(t, 6.283185307179586476925286766559);
        if (t <= -3.14159265358979323846) t += 6.283185307179586476925286766559;
        theta[2 * x + mu] = t;
      }
    }
  }
  if (accepted_out) *accepted_out = accepted;
}

/* U_x^mu = (cos theta, sin theta) interleaved: U[(2*x + mu)*2 + {0,1}]. */
void links_from_angles(int64_t nlinks, const double *theta, double *U) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nlinks; ++i) {
    U[2 * i] = cos(theta[i]);
    U[2 * i + 1] = sin(theta[i]);
  }
}

/* Random U(1) phases Omega_x = exp(i phi_x), phi uniform in [0, 2pi). */
void gen_u1_phases(int64_t nsites, uint64_t seed, uint64_t tag, double *omega) {
  uint32_t key[2];
  seed_key(seed, key);
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nsites; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)tag, (uint32_t)(tag >> 32)};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    double ua, ub;
    two_uniforms(w, &ua, &ub);
    omega[2 * i] = cos(two_pi * ub);
    omega[2 * i + 1] = sin(two_pi * ub);
  }
}

/* Number of OpenMP threads the generators use (1 without OpenMP). */
int gen_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* SU(3) gauge fields in 4d                                                  */
/* ------------------------------------------------------------------------ */
/*
 * A 3 x 3 complex matrix is 18 doubles, row-major, (re, im) interleaved.
 * Links: U[((x * 4 + mu) * 3 + a) * 3 + b], x = x0 + L0 (x1 + L1 (x2 + L2 x3)),
 * U_x^mu the link from x to x + mu-hat.
 */
typedef struct { double re, im; } cplx;

static inline cplx cx(double re, double im) { cplx z = {re, im}; return z; }
static inline cplx cadd(cplx a, cplx b) { return cx(a.re + b.re, a.im + b.im); }
static inline cplx csub(cplx a, cplx b) { return cx(a.re - b.re, a.im - b.im); }
static inline cplx cmul(cplx a, cplx b) { return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static inline cplx cconj(cplx a) { return cx(a.re, -a.im); }
static inline cplx cscale(double s, cplx a) { return cx(s * a.re, s * a.im); }

static inline cplx mget(const double *m, int a, int b) { return cx(m[(a * 3 + b) * 2], m[(a * 3 + b) * 2 + 1]); }
static inline void mset(double *m, int a, int b, cplx z) {
  m[(a * 3 + b) * 2] = z.re;
  m[(a * 3 + b) * 2 + 1] = z.im;
}

/*
 * Projection to SU(3): rows 1 and 2 made orthonormal by Gram-Schmidt (row 1
 * normalised, row 2 orthogonalised against it and normalised), row 3 set to
 * conj(row1 x row2), which gives det = 1.
 */
static void su3_project(double *m) {
  cplx r0[3], r1[3];
  double n0 = 0.0;
  for (int b = 0; b < 3; ++b) {
    r0[b] = mget(m, 0, b);
    n0 += r0[b].re * r0[b].re + r0[b].im * r0[b].im;
  }
  n0 = 1.0 / sqrt(n0);
  for (int b = 0; b < 3; ++b) r0[b] = cscale(n0, r0[b]);
  cplx dot = cx(0.0, 0.0); /* <r0, r1> = sum conj(r0) r1 */
  for (int b = 0; b < 3; ++b) {
    r1[b] = mget(m, 1, b);
    dot = cadd(dot, cmul(cconj(r0[b]), r1[b]));
  }
  double n1 = 0.0;
  for (int b = 0; b < 3; ++b) {
    r1[b] = csub(r1[b], cmul(dot, r0[b]));
    n1 += r1[b].re * r1[b].re + r1[b].im * r1[b].im;
  }
  n1 = 1.0 / sqrt(n1);
  for (int b = 0; b < 3; ++b) r1[b] = cscale(n1, r1[b]);
  for (int b = 0; b < 3; ++b) {
    mset(m, 0, b, r0[b]);
    mset(m, 1, b, r1[b]);
  }
  mset(m, 2, 0, cconj(csub(cmul(r0[1], r1[2]), cmul(r0[2], r1[1]))));
  mset(m, 2, 1, cconj(csub(cmul(r0[2], r1[0]), cmul(r0[0], r1[2]))));
  mset(m, 2, 2, cconj(csub(cmul(r0[0], r1[1]), cmul(r0[1], r1[0]))));
}

/* Two independent standard normals for matrix i, pair j: Box-Muller on one Philox block */
static inline void gauss2(uint32_t key[2], int64_t i, uint32_t j, uint64_t tag, double g[2]) {
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t ctr[4] = {(uint32_t)i, ((uint32_t)((uint64_t)i >> 32) << 8) | j, (uint32_t)tag, (uint32_t)(tag >> 32)};
  uint32_t w[4];
  philox4x32_10(ctr, key, w);
  double u1, u2;
  two_uniforms(w, &u1, &u2);
  const double rad = sqrt(-2.0 * log(u1));
  g[0] = rad * cos(two_pi * u2);
  g[1] = rad * sin(two_pi * u2);
}

/*
 * n SU(3) matrices, each the projection (su3_project) of 1 + eps H with H
 * traceless hermitian, H = (1/sqrt 2) sum_a c_a lambda_a over the Gell-Mann
 * matrices, c_a independent N(0, 1): off-diagonal entries have Re, Im ~
 * N(0, 1/2). Random numbers: key = seed, counter (i, pair j, tag).
 */
void gen_su3_near_identity(int64_t n, double eps, uint64_t seed, uint64_t tag, double *out) {
  uint32_t key[2];
  seed_key(seed, key);
  const double s2 = 0.70710678118654752440, s3 = 0.57735026918962576451;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double c[8];
    for (uint32_t j = 0; j < 4; ++j) gauss2(key, i, j, tag, c + 2 * j);
    double *m = out + i * 18;
    /* c[0..7] = c_1 .. c_8 */
    const cplx h01 = cx(s2 * c[0], -s2 * c[1]);
    const cplx h02 = cx(s2 * c[3], -s2 * c[4]);
    const cplx h12 = cx(s2 * c[5], -s2 * c[6]);
    const double h00 = s2 * (c[2] + s3 * c[7]);
    const double h11 = s2 * (-c[2] + s3 * c[7]);
    const double h22 = s2 * (-2.0 * s3 * c[7]);
    mset(m, 0, 0, cx(1.0 + eps * h00, 0.0));
    mset(m, 1, 1, cx(1.0 + eps * h11, 0.0));
    mset(m, 2, 2, cx(1.0 + eps * h22, 0.0));
    mset(m, 0, 1, cscale(eps, h01));
    mset(m, 1, 0, cscale(eps, cconj(h01)));
    mset(m, 0, 2, cscale(eps, h02));
    mset(m, 2, 0, cscale(eps, cconj(h02)));
    mset(m, 1, 2, cscale(eps, h12));
    mset(m, 2, 1, cscale(eps, cconj(h12)));
    su3_project(m);
  }
}

/*
 * n random SU(3) matrices: su3_project of a matrix with independent complex
 * Gaussian entries (row Gram-Schmidt of a Gaussian matrix; used for random
 * gauge transformations).
 */
void gen_su3_random(int64_t n, uint64_t seed, uint64_t tag, double *out) {
  uint32_t key[2];
  seed_key(seed, key);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double g[18];
    for (uint32_t j = 0; j < 9; ++j) gauss2(key, i, j, tag, g + 2 * j);
    double *m = out + i * 18;
    for (int e = 0; e < 18; ++e) m[e] = g[e];
    su3_project(m);
  }
}

static inline void mmul(const double *a, const double *b, double *c) { /* c = a b */
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      cplx s = cx(0.0, 0.0);
      for (int j = 0; j < 3; ++j) s = cadd(s, cmul(mget(a, i, j), mget(b, j, k)));
      mset(c, i, k, s);
    }
}
static inline void mmul_dag_right(const double *a, const double *b, double *c) { /* c = a b^dagger */
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      cplx s = cx(0.0, 0.0);
      for (int j = 0; j < 3; ++j) s = cadd(s, cmul(mget(a, i, j), cconj(mget(b, k, j))));
      mset(c, i, k, s);
    }
}
static inline void mmul_dag_left(const double *a, const double *b, double *c) { /* c = a^dagger b */
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      cplx s = cx(0.0, 0.0);
      for (int j = 0; j < 3; ++j) s = cadd(s, cmul(cconj(mget(a, j, i)), mget(b, j, k)));
      mset(c, i, k, s);
    }
}

static inline int64_t site4(const int L[4], const int c[4]) {
  return c[0] + (int64_t)L[0] * (c[1] + (int64_t)L[1] * (c[2] + (int64_t)L[2] * c[3]));
}

/*
 * One APE smearing step on a periodic 4d lattice, all links from the old
 * field (no ordering dependence): V = (1 - alpha) U_x^mu + (alpha / 6) S_x^mu,
 *   S_x^mu = sum_{nu != mu} [ U_x^nu U_{x+nu}^mu U_{x+mu}^nu^dagger
 *                           + U_{x-nu}^nu^dagger U_{x-nu}^mu U_{x-nu+mu}^nu ],
 * then Uout_x^mu = su3_project(V).
 */
void ape_smear_4d(const int L[4], double alpha, const double *Uin, double *Uout) {
  const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < V * 4; ++q) {
    const int64_t x = q / 4;
    const int mu = (int)(q % 4);
    int c[4];
    int64_t r = x;
    for (int k = 0; k < 4; ++k) {
      c[k] = (int)(r % L[k]);
      r /= L[k];
    }
    double S[18] = {0}, t1[18], t2[18];
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == mu) continue;
      int cp[4], cm[4], cpm[4], cmn[4];
      for (int k = 0; k < 4; ++k) cp[k] = cm[k] = cpm[k] = cmn[k] = c[k];
      cp[nu] = (c[nu] + 1) % L[nu];              /* x + nu */
      cm[mu] = (c[mu] + 1) % L[mu];              /* x + mu */
      cmn[nu] = (c[nu] - 1 + L[nu]) % L[nu];     /* x - nu */
      cpm[nu] = cmn[nu];
      cpm[mu] = (c[mu] + 1) % L[mu];             /* x - nu + mu */
      const double *Uxn = Uin + (x * 4 + nu) * 18;
      const double *Uxpn_mu = Uin + (site4(L, cp) * 4 + mu) * 18;
      const double *Uxpm_nu = Uin + (site4(L, cm) * 4 + nu) * 18;
      const double *Uxmn_nu = Uin + (site4(L, cmn) * 4 + nu) * 18;
      const double *Uxmn_mu = Uin + (site4(L, cmn) * 4 + mu) * 18;
      const double *Uxmnpm_nu = Uin + (site4(L, cpm) * 4 + nu) * 18;
      mmul(Uxn, Uxpn_mu, t1);
      mmul_dag_right(t1, Uxpm_nu, t2);
      for (int e = 0; e < 18; ++e) S[e] += t2[e];
      mmul_dag_left(Uxmn_nu, Uxmn_mu, t1);
      mmul(t1, Uxmnpm_nu, t2);
      for (int e = 0; e < 18; ++e) S[e] += t2[e];
    }
    double *o = Uout + q * 18;
    const double *u = Uin + q * 18;
    for (int e = 0; e < 18; ++e) o[e] = (1.0 - alpha) * u[e] + (alpha / 6.0) * S[e];
    su3_project(o);
  }
}
