/*
 * mond_oracle.c -- plain FP64 CPU oracle of the MOND particle-mesh method of
 * Visser, Eijt & de Nijs, "Fast particle-mesh code for Milgromian dynamics"
 * (A&A 2023, arXiv:2312.02968).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table
 * or constant generator with the CUDA library; the two only ever see the same
 * seeded inputs.
 *
 * Everything here is written for a reader checking it against the paper:
 * one loop per step, no blocking, no fusion. Floating point is FP64, except
 * where the fixed-point deposit rule defines integer arithmetic, and except
 * the FP32 density that rule defines as the deposit's output.
 *
 * Conventions (App. "Fourier transforms"):
 *   mesh index i in 0..n-1 on each axis, fields stored [z][y][x], x fastest;
 *   wave numbers k_a = 2*pi*m_a/L with m_a = i (i < n/2) or i-n (i >= n/2),
 *   so the Nyquist index n/2 carries k = -pi/s;
 *   forward  transform  f^(k) = s^3 * sum_r f(r) exp(-i k.r),
 *   inverse  transform  f(r)  = L^-3 * sum_k f^(k) exp(+i k.r).
 * Vector fields are three consecutive scalar planes (component-major).
 * Particles are triples [N][3]: integer cell (FFT-domain index) plus an FP32
 * offset in [-1/2, 1/2] pixels from that cell's centre, and a velocity.
 *
 * Pins (what fixes each function independently of itself; tests/test_oracle_*):
 *   ora_ball           251 taps at sigma = 1 (Sect. 3.1, Fig. 1); brute-force counts
 *   ora_axis_lut       Poisson-summation normalisation of the sampled Gaussian
 *   ora_deposit_fixed  direct FP64 Eq. smooth within the rule's error bound;
 *                      one-particle spectrum exp(-sigma^2 k^2 / 2) (App. Fourier);
 *                      mass conservation; independence of particle order
 *   ora_fft*           plain DFT, numpy.fft, round trip, Parseval
 *   ora_mu / ora_nu    mu(x) x = y <=> nu(y) y = x (Sect. 2.1)
 *   ora_solve          42 transforms for K = 4, 2 for Newton (Sect. 5.2, Sect. 6);
 *                      Newtonian closed form; spectral Poisson of a point mass;
 *                      curl/div invariants; deep-MOND point mass sqrt(GMa0)/r
 *                      (Sect. 2); Eq. twobodyforce; Eq. ringforce; Eq. g of the
 *                      isothermal sphere; low-k AQUAL residual falls tenfold in
 *                      three iterations; convergence rate (Sect. 2.1); the FP64
 *                      period-2 cycle at the zero of the field
 *   ora_aqual_solve    a fixed point of the iteration (odd grids); brute-force
 *                      minimisation of the same energy; Newtonian closed form
 *   ora_deposit_fixed  (integer rule) a hand-worked particle; every tap of single
 *                      particles recomputed from the rule
 *   ora_gather         node-smoothed field at nodes; constant field; two-body force
 *   ora_push           Eq. motion on hand-checked numbers
 *   ora_particle_diag  two-body constants of motion on hand-made states
 *   ora_solve_increment  Newtonian kind: equals the difference of two full
 *                      solves; linear in drho; central difference of the full
 *                      iteration about a converged base (error O(eps^2));
 *                      ora_linearised against central differences of nu/mu
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORA_OK 0
#define ORA_EINVAL -1
#define ORA_ENOMEM -2

enum { ORA_MU_DEEP = 0, ORA_MU_SIMPLE = 1, ORA_MU_STANDARD = 2, ORA_MU_NEWTON = 3 };

static long long g_transform_count = 0; /* scalar 3-D transforms, for the 42-FFT check */

long long ora_transform_count(void) { return g_transform_count; }
void ora_reset_transform_count(void) { g_transform_count = 0; }

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops from now on (timing of the oracle at a given
 * thread count); returns the count in force. */
int ora_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
  return omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}

static inline int64_t idx3(int n, int x, int y, int z) {
  return ((int64_t)z * n + y) * n + x;
}
static inline int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}
/* signed frequency index of array index i (App. Fourier: -n/2 .. n/2-1 for
 * even n; the symmetric range -(n-1)/2 .. (n-1)/2 for odd n) */
static inline int freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

/* ------------------------------------------------------------------------ */
/* Interpolation functions (Eq. mu, Sect. 2.1 pair mu/nu, Sect. 4 deep MOND)  */
/* ------------------------------------------------------------------------ */

/* mu(x): deep x; simple x/(1+x); standard x/sqrt(1+x^2) (Eq. mu); Newton 1. */
double ora_mu(int kind, double x) {
  switch (kind) {
    case ORA_MU_DEEP: return x;
    case ORA_MU_SIMPLE: return x / (1.0 + x);
    case ORA_MU_STANDARD: return x / sqrt(1.0 + x * x);
    default: return 1.0;
  }
}

/* nu(y), the inverse pair: mu(x) x = y  <=>  nu(y) y = x (Sect. 2.1).
 * deep 1/sqrt(y) (Sect. 4); simple 1/2 + sqrt(1/4 + 1/y);
 * standard sqrt(1/2 + 1/2 sqrt(1 + 4/y^2)) (Sect. 2.1). */
double ora_nu(int kind, double y) {
  switch (kind) {
    case ORA_MU_DEEP: return 1.0 / sqrt(y);
    case ORA_MU_SIMPLE: return 0.5 + sqrt(0.25 + 1.0 / y);
    case ORA_MU_STANDARD: return sqrt(0.5 + 0.5 * sqrt(1.0 + 4.0 / (y * y)));
    default: return 1.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Ball of taps (Sect. 3.1, Fig. 1; App. Flow init step 2)                    */
/* ------------------------------------------------------------------------ */

/* Largest per-axis reach r with r^2 < (4 sigma)^2. */
int ora_ball_reach(double sigma) {
  double lim = 16.0 * sigma * sigma;
  int r = 0;
  while ((double)((r + 1) * (r + 1)) < lim) r++;
  return r;
}

/* Offsets d with |d|^2 < (4 sigma)^2 (radius 4 pixels of width sigma; 251 for
 * sigma = 1). Written z-major, then y, then x. Returns the count, or the count
 * needed if cap is too small. */
int ora_ball(double sigma, int32_t* d, int cap) {
  double lim = 16.0 * sigma * sigma;
  int r = ora_ball_reach(sigma);
  int cnt = 0;
  for (int dz = -r; dz <= r; dz++)
    for (int dy = -r; dy <= r; dy++)
      for (int dx = -r; dx <= r; dx++) {
        if ((double)(dx * dx + dy * dy + dz * dz) < lim) {
          if (cnt < cap) {
            d[3 * cnt + 0] = dx;
            d[3 * cnt + 1] = dy;
            d[3 * cnt + 2] = dz;
          }
          cnt++;
        }
      }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Fixed-point deposit (Eq. smooth with the lookup table of Sect. 3.1 and    */
/* App. Flow init step 1; integer rule so that the sum is order-independent) */
/* ------------------------------------------------------------------------ */

#define ORA_QBITS 16
#define ORA_QHALF (1 << (ORA_QBITS - 1)) /* 32768 */
#define ORA_NQ ((1 << ORA_QBITS) + 1)    /* 65537 table rows */

/* One-dimensional Gaussian of width sigma pixels (the separable factor of
 * Eq. smooth): g1(u) = exp(-u^2/(2 sigma^2)) / (sigma sqrt(2 pi)). */
static double g1(double u, double sigma) {
  return exp(-(u * u) / (2.0 * sigma * sigma)) / (sigma * sqrt(2.0 * M_PI));
}

/* Table W[q + 32768][j] = round_half_even(2^24 g1((j - r) - q/2^16)) for
 * q in [-32768, 32768] and j in [0, 2r]. lut must hold 65537*(2r+1) words. */
void ora_axis_lut(double sigma, uint32_t* lut) {
  int r = ora_ball_reach(sigma);
  int w = 2 * r + 1;
  for (int qi = 0; qi < ORA_NQ; qi++) {
    int q = qi - ORA_QHALF;
    for (int j = 0; j < w; j++) {
      double u = (double)(j - r) - (double)q * (1.0 / 65536.0);
      double v = nearbyint(g1(u, sigma) * 16777216.0);
      lut[(int64_t)qi * w + j] = (uint32_t)v;
    }
  }
}

/* Offset quantisation: q = round_half_even(offset * 2^16). */
static int quant_offset(float off) { return (int)nearbyint((double)off * 65536.0); }

static int ceil_log2_i64(int64_t n) {
  int l = 0;
  while (((int64_t)1 << l) < n) l++;
  return l;
}

/* Accumulator scale exponent: acc units are 2^-Kacc mass units, chosen so that
 * N * max|m| * 2^Kacc <= 2^62 (every cell total then fits in int64 with room).
 * max|m| < 2^E with E = max(biased exponent, 1) - 126 over the FP32 masses. */
int ora_kacc(int64_t n, const float* mass) {
  int emax = 1;
  for (int64_t i = 0; i < n; i++) {
    uint32_t b;
    memcpy(&b, &mass[i], 4);
    int e = (int)((b >> 23) & 0xFF);
    if (e > emax) emax = e;
  }
  int E = emax - 126;
  int L = n > 0 ? ceil_log2_i64(n) : 0;
  return 62 - E - L;
}

/* Integer rule of one tap. Axis weights W (2^-24 units) come from the table.
 * The mass significand msig is folded into the x weights,
 *   MX[j]    = (Wx[j] msig + 2^15) >> 16,
 * the y and z weights are combined per row,
 *   R[dy,dz] = (Wy[dy] Wz[dz] + 2^15) >> 16,
 * and the tap's contribution is P = R MX (exact, < 2^62) shifted to 2^-Kacc
 * mass units with round-half-up: c = (P + 2^(sh-1)) >> sh, sh = 40 - Kacc - e2
 * where |m| = msig 2^e2. */
static uint64_t round_shift(uint64_t p, int sh) {
  if (p == 0) return 0;
  if (sh <= 0) return p << (-sh);
  if (sh >= 64) return 0;
  return (p + ((uint64_t)1 << (sh - 1))) >> sh;
}

/* Deposit of Eq. smooth on the periodic n^3 FFT domain, restricted to the ball
 * around each particle's cell, in the fixed-point rule above. acc (n^3 words,
 * int64 two's complement, cleared here) receives the sum; a particle whose
 * cell is outside [0,n) or whose offset is outside [-1/2, 1/2] or not finite
 * is skipped and counted in the return value. */
int64_t ora_deposit_fixed(int n, double sigma, int64_t N, const int32_t* cell,
                          const float* off, const float* mass, int kacc, uint64_t* acc) {
  int r = ora_ball_reach(sigma);
  int w = 2 * r + 1;
  int nb = ora_ball(sigma, NULL, 0);
  int32_t* ball = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)nb);
  uint32_t* lut = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)ORA_NQ * w);
  ora_ball(sigma, ball, nb);
  ora_axis_lut(sigma, lut);
  memset(acc, 0, sizeof(uint64_t) * (size_t)n * n * n);
  int64_t skipped = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : skipped)
  for (int64_t i = 0; i < N; i++) {
    int c[3];
    int q[3];
    int ok = 1;
    for (int a = 0; a < 3; a++) {
      c[a] = cell[3 * i + a];
      float o = off[3 * i + a];
      if (c[a] < 0 || c[a] >= n || !(o >= -0.5f && o <= 0.5f)) ok = 0;
      q[a] = ok ? quant_offset(o) : 0;
    }
    uint32_t b;
    memcpy(&b, &mass[i], 4);
    int eb = (int)((b >> 23) & 0xFF);
    if (eb == 0xFF) ok = 0;
    if (!ok) {
      skipped++;
      continue;
    }
    int neg = (int)(b >> 31);
    uint32_t msig = eb ? ((b & 0x7FFFFFu) | 0x800000u) : (b & 0x7FFFFFu);
    int e2 = eb ? eb - 150 : -149; /* |m| = msig * 2^e2 */
    int sh = 40 - kacc - e2;
    const uint32_t* Wx = lut + (int64_t)(q[0] + ORA_QHALF) * w;
    const uint32_t* Wy = lut + (int64_t)(q[1] + ORA_QHALF) * w;
    const uint32_t* Wz = lut + (int64_t)(q[2] + ORA_QHALF) * w;
    uint64_t MX[64], R[64][64];
    for (int j = 0; j < w; j++) MX[j] = ((uint64_t)Wx[j] * msig + 32768u) >> 16;
    for (int a = 0; a < w; a++)
      for (int b = 0; b < w; b++) R[a][b] = ((uint64_t)Wy[a] * Wz[b] + 32768u) >> 16;
    for (int t = 0; t < nb; t++) {
      int dx = ball[3 * t], dy = ball[3 * t + 1], dz = ball[3 * t + 2];
      uint64_t cval = round_shift(R[dy + r][dz + r] * MX[dx + r], sh);
      if (neg) cval = (uint64_t)0 - cval;
      int64_t j = idx3(n, wrap(c[0] + dx, n), wrap(c[1] + dy, n), wrap(c[2] + dz, n));
#pragma omp atomic
      acc[j] += cval;
    }
  }
  free(ball);
  free(lut);
  return skipped;
}

/* Density from the accumulator: rho = acc * 2^-Kacc / s^3, formed in FP64
 * (int64 -> double, one multiply by scale = 2^-Kacc/(s*s*s)), and also rounded
 * to FP32 (the deposit's defined output). Either output may be NULL. */
void ora_acc_to_rho(int n, const uint64_t* acc, int kacc, double s, float* rho32, double* rho64) {
  double scale = ldexp(1.0, -kacc) / (s * s * s);
  int64_t tot = (int64_t)n * n * n;
#pragma omp parallel for
  for (int64_t j = 0; j < tot; j++) {
    double v = (double)(int64_t)acc[j] * scale;
    if (rho32) rho32[j] = (float)v;
    if (rho64) rho64[j] = v;
  }
}

/* Eq. smooth evaluated directly in FP64 (exp per tap, no table, no
 * quantisation), over the same ball. Used to bound the fixed-point rule's
 * error. rho is cleared here. */
void ora_deposit_exact(int n, double sigma, double s, int64_t N, const int32_t* cell,
                       const float* off, const float* mass, double* rho) {
  int nb = ora_ball(sigma, NULL, 0);
  int32_t* ball = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)nb);
  ora_ball(sigma, ball, nb);
  memset(rho, 0, sizeof(double) * (size_t)n * n * n);
  double inv_s3 = 1.0 / (s * s * s);
  for (int64_t i = 0; i < N; i++) {
    for (int t = 0; t < nb; t++) {
      int d[3] = {ball[3 * t], ball[3 * t + 1], ball[3 * t + 2]};
      double w = 1.0;
      for (int a = 0; a < 3; a++) w *= g1((double)d[a] - (double)off[3 * i + a], sigma);
      int64_t j = idx3(n, wrap(cell[3 * i] + d[0], n), wrap(cell[3 * i + 1] + d[1], n),
                       wrap(cell[3 * i + 2] + d[2], n));
      rho[j] += (double)mass[i] * w * inv_s3;
    }
  }
  free(ball);
}

/* ------------------------------------------------------------------------ */
/* FFT: own mixed-radix recursive Cooley-Tukey (smallest prime factor first; */
/* a prime length falls through to the plain O(p^2) combination = naive DFT) */
/* ------------------------------------------------------------------------ */

/* Plain DFT by the definition, X[k] = sum_j x[j] exp(sign*2 pi i jk/n). */
void ora_dft1(int n, const cplx* x, cplx* X, int sign) {
  for (int k = 0; k < n; k++) {
    cplx acc = 0;
    for (int j = 0; j < n; j++) {
      double ang = sign * 2.0 * M_PI * (double)(((int64_t)j * k) % n) / (double)n;
      acc += x[j] * (cos(ang) + I * sin(ang));
    }
    X[k] = acc;
  }
}

static int smallest_factor(int n) {
  for (int p = 2; p * p <= n; p++)
    if (n % p == 0) return p;
  return n;
}

/* Recursive decimation in time: the length-n transform of in[0], in[stride],
 * ... is written to out[0..n-1]. tw[j] = exp(sign 2 pi i j/N) for the
 * top-level length N; this level uses every (N/n)-th entry. */
static void fft_rec(int n, const cplx* in, int stride, cplx* out, const cplx* tw, int N, cplx* scratch) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  int p = smallest_factor(n);
  int m = n / p;
  /* p interleaved sub-transforms of length m into out[q*m .. q*m+m-1] */
  for (int q = 0; q < p; q++) fft_rec(m, in + (int64_t)q * stride, stride * p, out + q * m, tw, N, scratch);
  int step = N / n;
  for (int k = 0; k < m; k++) {
    for (int q = 0; q < p; q++) scratch[q] = out[q * m + k];
    for (int j = 0; j < p; j++) {
      int kk = k + j * m; /* output index */
      cplx acc = 0;
      for (int q = 0; q < p; q++) acc += scratch[q] * tw[(int64_t)((q * kk) % n) * step];
      out[kk] = acc;
    }
  }
}

/* In-place 1-D transform of x[0], x[stride], ..., unnormalised. */
static void fft_line(int n, cplx* x, int64_t stride, int sign, const cplx* tw, cplx* buf, cplx* out, cplx* scratch) {
  for (int j = 0; j < n; j++) buf[j] = x[j * stride];
  fft_rec(n, buf, 1, out, tw, n, scratch);
  for (int j = 0; j < n; j++) x[j * stride] = out[j];
}

/* Unnormalised 1-D transform (exposed for the FFT pins). */
void ora_fft1(int n, cplx* x, int sign) {
  cplx* tw = (cplx*)malloc(sizeof(cplx) * n);
  cplx* buf = (cplx*)malloc(sizeof(cplx) * n);
  cplx* out = (cplx*)malloc(sizeof(cplx) * n);
  cplx* scr = (cplx*)malloc(sizeof(cplx) * n);
  for (int j = 0; j < n; j++) tw[j] = cos(sign * 2.0 * M_PI * j / n) + I * sin(sign * 2.0 * M_PI * j / n);
  fft_line(n, x, 1, sign, tw, buf, out, scr);
  free(tw);
  free(buf);
  free(out);
  free(scr);
}

/* Unnormalised 3-D transform of an n^3 array, one axis at a time. */
void ora_fft3_raw(int n, cplx* a, int sign) {
  cplx* tw = (cplx*)malloc(sizeof(cplx) * n);
  for (int j = 0; j < n; j++) tw[j] = cos(sign * 2.0 * M_PI * j / n) + I * sin(sign * 2.0 * M_PI * j / n);
  for (int axis = 0; axis < 3; axis++) {
    int64_t stride = axis == 0 ? 1 : (axis == 1 ? n : (int64_t)n * n);
#pragma omp parallel
    {
      cplx* buf = (cplx*)malloc(sizeof(cplx) * n);
      cplx* out = (cplx*)malloc(sizeof(cplx) * n);
      cplx* scr = (cplx*)malloc(sizeof(cplx) * n);
#pragma omp for
      for (int64_t line = 0; line < (int64_t)n * n; line++) {
        int u = (int)(line % n), v = (int)(line / n);
        int64_t base;
        if (axis == 0) base = idx3(n, 0, u, v);
        else if (axis == 1) base = idx3(n, u, 0, v);
        else base = idx3(n, u, v, 0);
        fft_line(n, a + base, stride, sign, tw, buf, out, scr);
      }
      free(buf);
      free(out);
      free(scr);
    }
  }
  free(tw);
}

/* Forward transform with the paper's normalisation: f^ = s^3 sum f e^{-ikr}. */
static void fwd3(int n, double s, cplx* a) {
  ora_fft3_raw(n, a, -1);
  double sc = s * s * s;
  int64_t tot = (int64_t)n * n * n;
  for (int64_t j = 0; j < tot; j++) a[j] *= sc;
  g_transform_count++;
}

/* Inverse with the paper's normalisation f = L^-3 sum f^ e^{ikr}; the real
 * part is kept (fields are real; see the Nyquist reading in the design notes). */
static void inv3_real(int n, double s, cplx* a, double* out) {
  ora_fft3_raw(n, a, +1);
  double L = n * s;
  double sc = 1.0 / (L * L * L);
  int64_t tot = (int64_t)n * n * n;
  for (int64_t j = 0; j < tot; j++) out[j] = creal(a[j]) * sc;
  g_transform_count++;
}

/* Wave vector k for array index (i, j, l) -> (kx, ky, kz), and A = 1/k.k with
 * A(0) = 0 (App. Flow init steps 3-4). */
static inline void kvec(int n, double s, int i, int j, int l, double* k) {
  double dk = 2.0 * M_PI / (n * s);
  k[0] = dk * freq(i, n);
  k[1] = dk * freq(j, n);
  k[2] = dk * freq(l, n);
}
static inline double invlap(const double* k) {
  double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  return kk > 0 ? 1.0 / kk : 0.0;
}

/* Periodic central finite difference, gradient component a of f:
 * (f[i+e_a] - f[i-e_a]) / (2 s). */
static void fd_grad(int n, double s, const double* f, double* g /* 3 planes */) {
  int64_t tot = (int64_t)n * n * n;
#pragma omp parallel for
  for (int z = 0; z < n; z++)
    for (int y = 0; y < n; y++)
      for (int x = 0; x < n; x++) {
        int64_t j = idx3(n, x, y, z);
        g[j] = (f[idx3(n, wrap(x + 1, n), y, z)] - f[idx3(n, wrap(x - 1, n), y, z)]) / (2.0 * s);
        g[tot + j] = (f[idx3(n, x, wrap(y + 1, n), z)] - f[idx3(n, x, wrap(y - 1, n), z)]) / (2.0 * s);
        g[2 * tot + j] = (f[idx3(n, x, y, wrap(z + 1, n))] - f[idx3(n, x, y, wrap(z - 1, n))]) / (2.0 * s);
      }
}

/* ------------------------------------------------------------------------ */
/* Field solve: App. Flow main-loop steps 3-9 (the iteration of Sect. 2.1)   */
/* ------------------------------------------------------------------------ */

/*
 * Inputs: rho (n^3, mass per s^3), n_iter = K (0 = Newtonian only),
 * H0 (3 n^3 or NULL = zero), finish_h (nonzero: the last iteration also runs
 * the mu, H and divergence-free steps, so that H is fresh for a warm start).
 * Outputs (any may be NULL): gN (3 n^3), H (3 n^3, the last H formed), phi
 * (n^3), acc = -grad_FD phi (3 n^3), dH (n_iter doubles: ||H_j - H_{j-1}||_2
 * over ||H_j||_2, NaN where no H was formed), gM (3 n^3: the curl-free g_M of
 * the last iteration, the point the mu step of an incremental solve is
 * linearised about).
 * For K = 0 the potential is phi_N and acc = g_N.
 */
int ora_solve_ex(int n, double s, double G, double a0, int mu_kind, int n_iter, const double* rho,
                 const double* H0, int finish_h, int mean_last2, double* gN_out, double* H_out, double* phi_out,
                 double* acc_out, double* dH_out, double* gM_out);

int ora_solve(int n, double s, double G, double a0, int mu_kind, int n_iter, const double* rho,
              const double* H0, int finish_h, double* gN_out, double* H_out, double* phi_out,
              double* acc_out, double* dH_out, double* gM_out) {
  return ora_solve_ex(n, s, G, a0, mu_kind, n_iter, rho, H0, finish_h, 0, gN_out, H_out, phi_out, acc_out, dH_out,
                      gM_out);
}

/* As ora_solve; with mean_last2 != 0 and n_iter >= 2 the potential of step 9
 * is the mean of the potentials of the last two iterations' curl-free steps,
 * phi^ = (phi^_{K-1} + phi^_K) / 2: the midpoint of the period-2 cycle the
 * iteration enters near zeros of the field (reading R14). */
int ora_solve_ex(int n, double s, double G, double a0, int mu_kind, int n_iter, const double* rho,
                 const double* H0, int finish_h, int mean_last2, double* gN_out, double* H_out, double* phi_out,
                 double* acc_out, double* dH_out, double* gM_out) {
  int64_t tot = (int64_t)n * n * n;
  cplx* c1 = (cplx*)malloc(sizeof(cplx) * tot);       /* scalar spectrum */
  cplx* cv = (cplx*)malloc(sizeof(cplx) * 3 * tot);   /* vector spectrum */
  double* gN = (double*)malloc(sizeof(double) * 3 * tot);
  double* H = (double*)malloc(sizeof(double) * 3 * tot);
  double* Hprev = (double*)malloc(sizeof(double) * 3 * tot);
  double* V = (double*)malloc(sizeof(double) * 3 * tot); /* F, then g_M */
  double* phi = (double*)malloc(sizeof(double) * tot);
  cplx* phih = (cplx*)malloc(sizeof(cplx) * tot);
  cplx* phih_prev = (mean_last2 && n_iter >= 2) ? (cplx*)malloc(sizeof(cplx) * tot) : NULL;
  if (!c1 || !cv || !gN || !H || !Hprev || !V || !phi || !phih || (mean_last2 && n_iter >= 2 && !phih_prev))
    return ORA_ENOMEM;

  /* step 3: rho^ = F(rho) */
  for (int64_t j = 0; j < tot; j++) c1[j] = rho[j];
  fwd3(n, s, c1);
  /* step 4: phi_N^ = -4 pi G A rho^ (sign: attractive gravity) */
  for (int l = 0; l < n; l++)
    for (int jy = 0; jy < n; jy++)
      for (int i = 0; i < n; i++) {
        double k[3];
        kvec(n, s, i, jy, l, k);
        int64_t j = idx3(n, i, jy, l);
        c1[j] = -4.0 * M_PI * G * invlap(k) * c1[j];
      }
  /* step 5: phi_N = F^-1(phi_N^) */
  inv3_real(n, s, c1, phi);
  /* step 6: g_N = -grad_FD phi_N */
  fd_grad(n, s, phi, gN);
  for (int64_t j = 0; j < 3 * tot; j++) gN[j] = -gN[j];

  if (n_iter == 0) {
    if (gN_out) memcpy(gN_out, gN, sizeof(double) * 3 * tot);
    if (phi_out) memcpy(phi_out, phi, sizeof(double) * tot);
    if (acc_out) memcpy(acc_out, gN, sizeof(double) * 3 * tot);
    if (H_out) memset(H_out, 0, sizeof(double) * 3 * tot);
    free(c1); free(cv); free(gN); free(H); free(Hprev); free(V); free(phi); free(phih);
    return ORA_OK;
  }

  /* step 7: F = g_N + H with H = H0 (0 by default) */
  if (H0) memcpy(H, H0, sizeof(double) * 3 * tot);
  else memset(H, 0, sizeof(double) * 3 * tot);

  for (int it = 1; it <= n_iter; it++) {
    /* F = g_N + H (Eq. helmholtz), then g_M = nu(|F|/a0) F (Eq. inverse) */
    for (int64_t j = 0; j < tot; j++) {
      double F[3], Fm = 0;
      for (int a = 0; a < 3; a++) {
        F[a] = gN[a * tot + j] + H[a * tot + j];
        Fm += F[a] * F[a];
      }
      Fm = sqrt(Fm);
      double f = Fm > 0 ? ora_nu(mu_kind, Fm / a0) : 0.0;
      for (int a = 0; a < 3; a++) V[a * tot + j] = f * F[a];
    }
    /* g_M^ = F(g_M) */
    for (int a = 0; a < 3; a++) {
      for (int64_t j = 0; j < tot; j++) cv[a * tot + j] = V[a * tot + j];
      fwd3(n, s, cv + a * tot);
    }
    /* phi^ = i A k.g_M^ ; g_M^ = -i k phi^ (curl-free part, Eq. rotg) */
    for (int l = 0; l < n; l++)
      for (int jy = 0; jy < n; jy++)
        for (int i = 0; i < n; i++) {
          double k[3];
          kvec(n, s, i, jy, l, k);
          int64_t j = idx3(n, i, jy, l);
          double A = invlap(k);
          cplx kg = k[0] * cv[j] + k[1] * cv[tot + j] + k[2] * cv[2 * tot + j];
          cplx ph = I * A * kg;
          phih[j] = ph;
          for (int a = 0; a < 3; a++) cv[a * tot + j] = -I * k[a] * ph;
        }
    if (phih_prev && it == n_iter - 1) memcpy(phih_prev, phih, sizeof(cplx) * tot);
    if (it == n_iter && !finish_h) {
      if (dH_out) dH_out[it - 1] = NAN;
      if (gM_out)
        for (int a = 0; a < 3; a++) inv3_real(n, s, cv + a * tot, gM_out + a * tot);
      break;
    }
    /* g_M = F^-1(g_M^) */
    for (int a = 0; a < 3; a++) inv3_real(n, s, cv + a * tot, V + a * tot);
    if (it == n_iter && gM_out) memcpy(gM_out, V, sizeof(double) * 3 * tot);
    /* F = mu(|g_M|/a0) g_M (Eq. interpolation); H = F - g_N (Eq. helmholtz) */
    memcpy(Hprev, H, sizeof(double) * 3 * tot);
    for (int64_t j = 0; j < tot; j++) {
      double gm = 0;
      for (int a = 0; a < 3; a++) gm += V[a * tot + j] * V[a * tot + j];
      gm = sqrt(gm);
      double f = ora_mu(mu_kind, gm / a0);
      for (int a = 0; a < 3; a++) H[a * tot + j] = f * V[a * tot + j] - gN[a * tot + j];
    }
    /* H^ = F(H); H^ -> H^ - k A k.H^ (divergence-free part, Eq. divH) */
    for (int a = 0; a < 3; a++) {
      for (int64_t j = 0; j < tot; j++) cv[a * tot + j] = H[a * tot + j];
      fwd3(n, s, cv + a * tot);
    }
    for (int l = 0; l < n; l++)
      for (int jy = 0; jy < n; jy++)
        for (int i = 0; i < n; i++) {
          double k[3];
          kvec(n, s, i, jy, l, k);
          int64_t j = idx3(n, i, jy, l);
          double A = invlap(k);
          cplx kh = k[0] * cv[j] + k[1] * cv[tot + j] + k[2] * cv[2 * tot + j];
          for (int a = 0; a < 3; a++) cv[a * tot + j] -= k[a] * A * kh;
        }
    /* H = F^-1(H^) */
    for (int a = 0; a < 3; a++) inv3_real(n, s, cv + a * tot, H + a * tot);
    if (dH_out) {
      double num = 0, den = 0;
      for (int64_t j = 0; j < 3 * tot; j++) {
        double d = H[j] - Hprev[j];
        num += d * d;
        den += H[j] * H[j];
      }
      dH_out[it - 1] = den > 0 ? sqrt(num / den) : 0.0;
    }
  }
  if (phih_prev)
    for (int64_t j = 0; j < tot; j++) phih[j] = 0.5 * (phih[j] + phih_prev[j]);
  /* step 9: phi = F^-1(phi^); acceleration mesh = -grad_FD phi (Sect. 3.2) */
  inv3_real(n, s, phih, phi);
  if (acc_out) {
    fd_grad(n, s, phi, acc_out);
    for (int64_t j = 0; j < 3 * tot; j++) acc_out[j] = -acc_out[j];
  }
  if (gN_out) memcpy(gN_out, gN, sizeof(double) * 3 * tot);
  if (H_out) memcpy(H_out, H, sizeof(double) * 3 * tot);
  if (phi_out) memcpy(phi_out, phi, sizeof(double) * tot);
  free(c1); free(cv); free(gN); free(H); free(Hprev); free(V); free(phi); free(phih); free(phih_prev);
  return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Incremental solve: the linearised nu and mu steps of Sect. 5.2 (v)        */
/* ------------------------------------------------------------------------ */

/* y nu'(y) and x mu'(x) for each kind (derivatives of the functions above):
 * deep      y nu' = -1/(2 sqrt y)                 x mu' = x
 * simple    y nu' = -1/(2 y sqrt(1/4 + 1/y))      x mu' = x/(1+x)^2
 * standard  y nu' = -1/(nu(y) y sqrt(y^2 + 4))    x mu' = x/(1+x^2)^(3/2)
 * Newton    0                                     0 */
double ora_ynu_prime(int kind, double y) {
  switch (kind) {
    case ORA_MU_DEEP: return -0.5 / sqrt(y);
    case ORA_MU_SIMPLE: return -1.0 / (2.0 * y * sqrt(0.25 + 1.0 / y));
    case ORA_MU_STANDARD: return -1.0 / (ora_nu(kind, y) * y * sqrt(y * y + 4.0));
    default: return 0.0;
  }
}
double ora_xmu_prime(int kind, double x) {
  switch (kind) {
    case ORA_MU_DEEP: return x;
    case ORA_MU_SIMPLE: return x / ((1.0 + x) * (1.0 + x));
    case ORA_MU_STANDARD: return x / pow(1.0 + x * x, 1.5);
    default: return 0.0;
  }
}

/* Linearisation of v -> f(|v|/a0) v about the point P, applied to dv:
 * f(p) dv + f'(p) (P.dv)/(a0 |P|) P = f(p) dv + p f'(p) (u.dv) u, with
 * p = |P|/a0 and u = P/|P| (Sect. 5.2 (v)). The identity for the Newtonian
 * kind; 0 where P = 0 otherwise (the zero-field reading of the nu step).
 * which = 0: f = nu; 1: f = mu. */
void ora_linearised(int kind, int which, double a0, const double* P, const double* dv, double* out) {
  double m = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
  if (kind == ORA_MU_NEWTON || !(m > 0)) {
    for (int a = 0; a < 3; a++) out[a] = kind == ORA_MU_NEWTON ? dv[a] : 0.0;
    return;
  }
  double p = m / a0;
  double f = which == 0 ? ora_nu(kind, p) : ora_mu(kind, p);
  double fp = which == 0 ? ora_ynu_prime(kind, p) : ora_xmu_prime(kind, p);
  double ud = (P[0] * dv[0] + P[1] * dv[1] + P[2] * dv[2]) / m;
  for (int a = 0; a < 3; a++) out[a] = f * dv[a] + fp * ud * P[a] / m;
}

/*
 * Incremental field solve (Sect. 5.2 (v)): the increments of the fields for a
 * density increment drho about a base state (g_N0, H0, g_M0), with the nu and
 * mu steps linearised about F0 = g_N0 + H0 and g_M0:
 *   dg_N = Newton(drho)                       (App. Flow steps 3-6)
 *   dH = 0; for j = 1..K:
 *     dF   = dg_N + dH
 *     dg_M = Jnu(F0) dF,  curl-free part      (Eq. inverse linearised, Eq. rotg)
 *     dF   = Jmu(g_M0) dg_M                   (Eq. interpolation linearised)
 *     dH   = div-free part of dF - dg_N       (Eq. helmholtz, Eq. divH)
 *   dphi^ = i A k.dg_M^ of the last iteration; dacc = -grad_FD dphi
 * The last iteration always finishes dH, so that the base can be moved on:
 * g_N1 = g_N0 + dg_N, H1 = H0 + dH, g_M1 = g_M0 + dg_M, acc1 = acc0 + dacc.
 * Outputs (any may be NULL): dgN, dH, dgM (the last curl-free dg_M), dacc,
 * all 3 n^3. n_iter >= 1.
 */
int ora_solve_increment(int n, double s, double G, double a0, int mu_kind, int n_iter, const double* drho,
                        const double* gN0, const double* H0, const double* gM0, double* dgN_out,
                        double* dH_out, double* dgM_out, double* dacc_out) {
  if (n_iter < 1) return ORA_EINVAL;
  int64_t tot = (int64_t)n * n * n;
  cplx* c1 = (cplx*)malloc(sizeof(cplx) * tot);
  cplx* cv = (cplx*)malloc(sizeof(cplx) * 3 * tot);
  double* dgN = (double*)malloc(sizeof(double) * 3 * tot);
  double* dH = (double*)calloc(3 * tot, sizeof(double));
  double* V = (double*)malloc(sizeof(double) * 3 * tot);
  double* phi = (double*)malloc(sizeof(double) * tot);
  cplx* phih = (cplx*)malloc(sizeof(cplx) * tot);
  if (!c1 || !cv || !dgN || !dH || !V || !phi || !phih) return ORA_ENOMEM;

  /* dg_N = -grad_FD F^-1(-4 pi G A F(drho)) */
  for (int64_t j = 0; j < tot; j++) c1[j] = drho[j];
  fwd3(n, s, c1);
  for (int l = 0; l < n; l++)
    for (int jy = 0; jy < n; jy++)
      for (int i = 0; i < n; i++) {
        double k[3];
        kvec(n, s, i, jy, l, k);
        int64_t j = idx3(n, i, jy, l);
        c1[j] = -4.0 * M_PI * G * invlap(k) * c1[j];
      }
  inv3_real(n, s, c1, phi);
  fd_grad(n, s, phi, dgN);
  for (int64_t j = 0; j < 3 * tot; j++) dgN[j] = -dgN[j];

  for (int it = 1; it <= n_iter; it++) {
    /* dg_M = Jnu(F0) (dg_N + dH) */
    for (int64_t j = 0; j < tot; j++) {
      double F0[3], dF[3], o[3];
      for (int a = 0; a < 3; a++) {
        F0[a] = gN0[a * tot + j] + H0[a * tot + j];
        dF[a] = dgN[a * tot + j] + dH[a * tot + j];
      }
      ora_linearised(mu_kind, 0, a0, F0, dF, o);
      for (int a = 0; a < 3; a++) V[a * tot + j] = o[a];
    }
    /* curl-free part; the potential increment of this iteration */
    for (int a = 0; a < 3; a++) {
      for (int64_t j = 0; j < tot; j++) cv[a * tot + j] = V[a * tot + j];
      fwd3(n, s, cv + a * tot);
    }
    for (int l = 0; l < n; l++)
      for (int jy = 0; jy < n; jy++)
        for (int i = 0; i < n; i++) {
          double k[3];
          kvec(n, s, i, jy, l, k);
          int64_t j = idx3(n, i, jy, l);
          double A = invlap(k);
          cplx kg = k[0] * cv[j] + k[1] * cv[tot + j] + k[2] * cv[2 * tot + j];
          cplx ph = I * A * kg;
          phih[j] = ph;
          for (int a = 0; a < 3; a++) cv[a * tot + j] = -I * k[a] * ph;
        }
    for (int a = 0; a < 3; a++) inv3_real(n, s, cv + a * tot, V + a * tot);
    if (it == n_iter && dgM_out) memcpy(dgM_out, V, sizeof(double) * 3 * tot);
    /* dH = div-free part of Jmu(g_M0) dg_M - dg_N */
    for (int64_t j = 0; j < tot; j++) {
      double P[3], dv[3], o[3];
      for (int a = 0; a < 3; a++) {
        P[a] = gM0[a * tot + j];
        dv[a] = V[a * tot + j];
      }
      ora_linearised(mu_kind, 1, a0, P, dv, o);
      for (int a = 0; a < 3; a++) dH[a * tot + j] = o[a] - dgN[a * tot + j];
    }
    for (int a = 0; a < 3; a++) {
      for (int64_t j = 0; j < tot; j++) cv[a * tot + j] = dH[a * tot + j];
      fwd3(n, s, cv + a * tot);
    }
    for (int l = 0; l < n; l++)
      for (int jy = 0; jy < n; jy++)
        for (int i = 0; i < n; i++) {
          double k[3];
          kvec(n, s, i, jy, l, k);
          int64_t j = idx3(n, i, jy, l);
          double A = invlap(k);
          cplx kh = k[0] * cv[j] + k[1] * cv[tot + j] + k[2] * cv[2 * tot + j];
          for (int a = 0; a < 3; a++) cv[a * tot + j] -= k[a] * A * kh;
        }
    for (int a = 0; a < 3; a++) inv3_real(n, s, cv + a * tot, dH + a * tot);
  }
  /* dacc = -grad_FD F^-1(dphi^) */
  inv3_real(n, s, phih, phi);
  if (dacc_out) {
    fd_grad(n, s, phi, dacc_out);
    for (int64_t j = 0; j < 3 * tot; j++) dacc_out[j] = -dacc_out[j];
  }
  if (dgN_out) memcpy(dgN_out, dgN, sizeof(double) * 3 * tot);
  if (dH_out) memcpy(dH_out, dH, sizeof(double) * 3 * tot);
  free(c1); free(cv); free(dgN); free(dH); free(V); free(phi); free(phih);
  return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Force at the particles (Eq. gi) and Leapfrog (Eq. motion)                  */
/* ------------------------------------------------------------------------ */

/* g_i = sum over the ball around the particle's cell of acc(x_p) times the
 * Gaussian of Eq. smooth at x_p - r_i (the pixel sum of Eq. gi; the s^3 of the
 * Riemann sum cancels the s^-3 of the normalisation). FP64 weights. */
void ora_gather(int n, double sigma, const double* acc, int64_t N, const int32_t* cell,
                const float* off, double* g) {
  int nb = ora_ball(sigma, NULL, 0);
  int32_t* ball = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)nb);
  ora_ball(sigma, ball, nb);
  int64_t tot = (int64_t)n * n * n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    double s3[3] = {0, 0, 0};
    for (int t = 0; t < nb; t++) {
      int d[3] = {ball[3 * t], ball[3 * t + 1], ball[3 * t + 2]};
      double w = 1.0;
      for (int a = 0; a < 3; a++) w *= g1((double)d[a] - (double)off[3 * i + a], sigma);
      int64_t j = idx3(n, wrap(cell[3 * i] + d[0], n), wrap(cell[3 * i + 1] + d[1], n),
                       wrap(cell[3 * i + 2] + d[2], n));
      for (int a = 0; a < 3; a++) s3[a] += acc[a * tot + j] * w;
    }
    for (int a = 0; a < 3; a++) g[3 * i + a] = s3[a];
  }
  free(ball);
}

/* Leapfrog kick then drift (Eq. motion): v += g dt; r += v dt. Positions are
 * kept as cell + offset in pixels; after the drift the cell is the nearest
 * pixel centre (offset in [-1/2, 1/2)) and wraps periodically. */
void ora_push(int n, double s, double dt, int64_t N, const double* g, int32_t* cell, double* off,
              double* vel, int drift) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    for (int a = 0; a < 3; a++) {
      vel[3 * i + a] += g[3 * i + a] * dt;
      if (!drift) continue;
      double x = (double)cell[3 * i + a] + off[3 * i + a] + vel[3 * i + a] * dt / s;
      double c = floor(x + 0.5);
      off[3 * i + a] = x - c;
      cell[3 * i + a] = wrap((int)c, n);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (the monitored quantities of Sects. 4.1 and 4.3)              */
/* ------------------------------------------------------------------------ */

/* out[0] mass, out[1..3] momentum P, out[4..6] centre of mass R,
 * out[7..9] angular momentum about R, out[10] kinetic energy.
 * Physical position x = (cell - n/2 + offset) s (App. Fourier grid). */
void ora_particle_diag(int n, double s, int64_t N, const int32_t* cell, const double* off,
                       const double* vel, const float* mass, double* out) {
  double M = 0, P[3] = {0, 0, 0}, R[3] = {0, 0, 0}, E = 0;
  for (int64_t i = 0; i < N; i++) {
    double m = mass[i];
    M += m;
    for (int a = 0; a < 3; a++) {
      double x = ((double)cell[3 * i + a] - n / 2 + off[3 * i + a]) * s;
      P[a] += m * vel[3 * i + a];
      R[a] += m * x;
      E += 0.5 * m * vel[3 * i + a] * vel[3 * i + a];
    }
  }
  for (int a = 0; a < 3; a++) R[a] = M > 0 ? R[a] / M : 0.0;
  double L[3] = {0, 0, 0};
  for (int64_t i = 0; i < N; i++) {
    double m = mass[i], x[3];
    for (int a = 0; a < 3; a++) x[a] = ((double)cell[3 * i + a] - n / 2 + off[3 * i + a]) * s - R[a];
    const double* v = vel + 3 * i;
    L[0] += m * (x[1] * v[2] - x[2] * v[1]);
    L[1] += m * (x[2] * v[0] - x[0] * v[2]);
    L[2] += m * (x[0] * v[1] - x[1] * v[0]);
  }
  out[0] = M;
  for (int a = 0; a < 3; a++) {
    out[1 + a] = P[a];
    out[4 + a] = R[a];
    out[7 + a] = L[a];
  }
  out[10] = E;
}

/* Divergence-free part of a vector field (Eq. divH): H^ -> H^ - k A k.H^,
 * k = 0 kept; the real part of the inverse transform is kept. */
void ora_project_div(int n, double s, const double* in, double* out) {
  int64_t tot = (int64_t)n * n * n;
  cplx* cv = (cplx*)malloc(sizeof(cplx) * 3 * tot);
  for (int64_t j = 0; j < 3 * tot; j++) cv[j] = in[j];
  for (int a = 0; a < 3; a++) fwd3(n, s, cv + a * tot);
  for (int l = 0; l < n; l++)
    for (int jy = 0; jy < n; jy++)
      for (int i = 0; i < n; i++) {
        double k[3];
        kvec(n, s, i, jy, l, k);
        int64_t j = idx3(n, i, jy, l);
        double A = invlap(k);
        cplx kh = k[0] * cv[j] + k[1] * cv[tot + j] + k[2] * cv[2 * tot + j];
        for (int a = 0; a < 3; a++) cv[a * tot + j] -= k[a] * A * kh;
      }
  for (int a = 0; a < 3; a++) inv3_real(n, s, cv + a * tot, out + a * tot);
  free(cv);
}

/* ------------------------------------------------------------------------ */
/* Apparent density and enclosed mass (Eq. apparentdensity, Eq. totalmass)   */
/* ------------------------------------------------------------------------ */

/* rho = -(div g) / (4 pi G), the divergence taken with the periodic central
 * difference of the gradient (f[i+1] - f[i-1]) / (2 s) on each axis.
 * g_N gives the baryonic density rho_B, the MOND acceleration the apparent
 * density rho_A. g: 3 planes (x, y, z components); rho: 1 plane. */
void ora_field_density(int n, double s, double G, const double* g, double* rho) {
  int64_t tot = (int64_t)n * n * n;
  double c = -1.0 / (4.0 * M_PI * G);
#pragma omp parallel for
  for (int z = 0; z < n; z++)
    for (int y = 0; y < n; y++)
      for (int x = 0; x < n; x++) {
        double dx = (g[idx3(n, wrap(x + 1, n), y, z)] - g[idx3(n, wrap(x - 1, n), y, z)]) / (2.0 * s);
        double dy = (g[tot + idx3(n, x, wrap(y + 1, n), z)] - g[tot + idx3(n, x, wrap(y - 1, n), z)]) / (2.0 * s);
        double dz = (g[2 * tot + idx3(n, x, y, wrap(z + 1, n))] - g[2 * tot + idx3(n, x, y, wrap(z - 1, n))]) /
                    (2.0 * s);
        rho[idx3(n, x, y, z)] = c * (dx + dy + dz);
      }
}

/* Mass inside the box W of cells lo..hi (inclusive on each axis, periodic)
 * from the outward flux of g through its six faces:
 * M(W) = -(1/(4 pi G)) sum over faces of g.dS. On a face the normal
 * component is the mean of the two cells the face separates, the face value
 * that the central-difference divergence implies, so M(W) equals the sum of
 * ora_field_density over W times s^3. */
double ora_box_flux_mass(int n, double s, double G, const double* g, const int32_t* lo, const int32_t* hi) {
  int64_t tot = (int64_t)n * n * n;
  double flux = 0.0;
  for (int a = 0; a < 3; a++) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    for (int side = 0; side < 2; side++) {
      /* the two cells straddling the face, along axis a */
      int in_a = side ? hi[a] : lo[a];
      int out_a = side ? hi[a] + 1 : lo[a] - 1;
      double sgn = side ? 1.0 : -1.0;
      for (int ib = lo[b]; ib <= hi[b]; ib++)
        for (int ic = lo[c]; ic <= hi[c]; ic++) {
          int p[3], q[3];
          p[a] = wrap(in_a, n);
          q[a] = wrap(out_a, n);
          p[b] = q[b] = wrap(ib, n);
          p[c] = q[c] = wrap(ic, n);
          double gin = g[a * tot + idx3(n, p[0], p[1], p[2])];
          double gout = g[a * tot + idx3(n, q[0], q[1], q[2])];
          flux += sgn * 0.5 * (gin + gout) * s * s;
        }
    }
  }
  return -flux / (4.0 * M_PI * G);
}

/* Mass in spherical shells about the point c (physical coordinates, cell i
 * at (i - n/2) s): out[k] += rho s^3 over the cells whose centre lies at a
 * minimum-image distance r with floor(r / dr) = k, for k < nbins. */
void ora_shell_mass(int n, double s, const double* rho, const double* c, double dr, int nbins, double* out) {
  double L = n * s;
  for (int k = 0; k < nbins; k++) out[k] = 0.0;
  for (int z = 0; z < n; z++)
    for (int y = 0; y < n; y++)
      for (int x = 0; x < n; x++) {
        double d[3];
        int ii[3] = {x, y, z};
        for (int a = 0; a < 3; a++) {
          d[a] = (ii[a] - n / 2) * s - c[a];
          d[a] -= L * nearbyint(d[a] / L);
        }
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double fk = floor(r / dr);
        if (fk < nbins) out[(int)fk] += rho[idx3(n, x, y, z)] * s * s * s;
      }
}

/* ------------------------------------------------------------------------ */
/* Mesh-interpolating gather: the node-smoothed acceleration (the force Eq.  */
/* gi gives a particle on each pixel centre) interpolated at the particles.  */
/* ------------------------------------------------------------------------ */

/* Interpolation weights along one axis for a particle at fraction t in [0, 1)
 * past node b. order 1: linear, nodes b, b+1. order 3: Keys' cubic
 * convolution kernel with a = -1/2, nodes b-1 .. b+2:
 *   W(x) = 1.5|x|^3 - 2.5|x|^2 + 1             for |x| <= 1,
 *   W(x) = -0.5|x|^3 + 2.5|x|^2 - 4|x| + 2     for 1 < |x| < 2. */
static double keys(double x) {
  x = fabs(x);
  if (x <= 1.0) return 1.5 * x * x * x - 2.5 * x * x + 1.0;
  if (x < 2.0) return -0.5 * x * x * x + 2.5 * x * x - 4.0 * x + 2.0;
  return 0.0;
}

/* g_i = sum over the interpolation nodes of the product of the per-axis
 * weights times S at the node (periodic). The particle sits at cell + off
 * (pixel units); the node below it is b = cell - 1 when off < 0, else cell.
 * S: 3 planes; out: [N][3]. */
void ora_interp_gather(int n, int order, const double* S, int64_t N, const int32_t* cell, const double* off,
                       double* out) {
  int64_t tot = (int64_t)n * n * n;
  int lo = order == 3 ? -1 : 0, hi = order == 3 ? 2 : 1;
#pragma omp parallel for
  for (int64_t i = 0; i < N; i++) {
    int b[3];
    double w[3][4];
    for (int a = 0; a < 3; a++) {
      double o = off[3 * i + a];
      b[a] = cell[3 * i + a] + (o < 0 ? -1 : 0);
      double t = o < 0 ? o + 1.0 : o;
      for (int j = lo; j <= hi; j++) w[a][j - lo] = order == 3 ? keys(t - j) : (j == 0 ? 1.0 - t : t);
    }
    double g[3] = {0, 0, 0};
    for (int dz = lo; dz <= hi; dz++)
      for (int dy = lo; dy <= hi; dy++)
        for (int dx = lo; dx <= hi; dx++) {
          double wt = w[0][dx - lo] * w[1][dy - lo] * w[2][dz - lo];
          int64_t j = idx3(n, wrap(b[0] + dx, n), wrap(b[1] + dy, n), wrap(b[2] + dz, n));
          for (int a = 0; a < 3; a++) g[a] += wt * S[a * tot + j];
        }
    for (int a = 0; a < 3; a++) out[3 * i + a] = g[a];
  }
}

/* ------------------------------------------------------------------------ */
/* Exact solution of the discretised AQUAL equation (Sect. 2.1, Eq. PDE)     */
/* ------------------------------------------------------------------------ */

/*
 * The iteration of Sect. 2.1 stops at its K-th iterate; this function finds
 * the field that iteration would reach if it converged: the potential phi
 * whose spectral gradient u = D phi satisfies the AQUAL equation on the mesh,
 *
 *   D^T [ mu(|u|/a0) u + g_N ] = 0,           (div of mu(|g|/a0) g = div g_N)
 *
 * with g = -u the MOND acceleration and g_N the Newtonian field of the
 * solve (App. Flow steps 3-6, here from ora_solve with K = 0). D_a is the
 * spectral derivative i k_a with the Nyquist term dropped (the real-part
 * convention of the odd operators), D^T its transpose (-div). The equation
 * is the stationarity condition of the convex energy
 *
 *   E(phi) = sum_cells [ a0^2 Psi(|D phi|/a0) + g_N . D phi ],
 *   Psi(x) = integral_0^x mu(t) t dt,
 *
 * (the mesh form of the AQUAL Lagrangian), whose gradient is
 * D^T [mu(|u|/a0) u + g_N]. Psi is convex for every interpolation function
 * here (x mu(x) increases), so E has one minimiser up to a constant in phi.
 * It is found by limited-memory BFGS (8 pairs) with the inverse spectral
 * Laplacian (D^T D)^-1 as the initial inverse Hessian and an Armijo
 * backtracking line search, starting from phi0 (NULL: zero), until
 * |grad E| <= tol |D^T g_N| or the line search can no longer lower E.
 * Outputs: phi (n^3), acc = -grad_FD phi (3 n^3, the acceleration mesh the
 * method would form from it, App. Flow step 9), info[0] = iterations,
 * info[1] = final relative gradient, info[2] = energy evaluations.
 */
static double psi_mu(int kind, double x) {
  double x2 = x * x;
  switch (kind) {
    case ORA_MU_DEEP: return x2 * x / 3.0;
    case ORA_MU_SIMPLE: /* x^2/2 - x + ln(1+x), by its series where that cancels */
      if (x < 1e-2) return x2 * x * (1.0 / 3.0 - x / 4.0 + x2 / 5.0 - x2 * x / 6.0 + x2 * x2 / 7.0);
      return 0.5 * x2 - x + log1p(x);
    case ORA_MU_STANDARD: /* (x sqrt(1+x^2) - asinh x) / 2 */
      if (x < 1e-2) return x2 * x * (1.0 / 3.0 - x2 / 10.0 + 3.0 * x2 * x2 / 56.0);
      return 0.5 * (x * sqrt(1.0 + x2) - asinh(x));
    case ORA_MU_NEWTON: return 0.5 * x2;
  }
  return NAN;
}

/* The wave number of odd operators: k_a, with 0 on axis a's Nyquist index. */
static inline void kvec_odd(int n, double s, int i, int j, int l, double* k) {
  kvec(n, s, i, j, l, k);
  if (n % 2 == 0) {
    if (i == n / 2) k[0] = 0.0;
    if (j == n / 2) k[1] = 0.0;
    if (l == n / 2) k[2] = 0.0;
  }
}

/* u = D phi (3 planes). c: n^3 complex scratch. */
static void aq_grad(int n, double s, const double* phi, double* u, cplx* c, cplx* c2) {
  int64_t tot = (int64_t)n * n * n;
  for (int64_t j = 0; j < tot; j++) c[j] = phi[j];
  fwd3(n, s, c);
  for (int a = 0; a < 3; a++) {
#pragma omp parallel for
    for (int l = 0; l < n; l++)
      for (int jy = 0; jy < n; jy++)
        for (int i = 0; i < n; i++) {
          double k[3];
          kvec_odd(n, s, i, jy, l, k);
          int64_t j = idx3(n, i, jy, l);
          c2[j] = I * k[a] * c[j];
        }
    inv3_real(n, s, c2, u + a * tot);
  }
}

/* out = D^T w = -sum_a D_a w_a (w: 3 planes). */
static void aq_gradT(int n, double s, const double* w, double* out, cplx* c, cplx* c2) {
  int64_t tot = (int64_t)n * n * n;
  for (int64_t j = 0; j < tot; j++) c2[j] = 0;
  for (int a = 0; a < 3; a++) {
    for (int64_t j = 0; j < tot; j++) c[j] = w[a * tot + j];
    fwd3(n, s, c);
#pragma omp parallel for
    for (int l = 0; l < n; l++)
      for (int jy = 0; jy < n; jy++)
        for (int i = 0; i < n; i++) {
          double k[3];
          kvec_odd(n, s, i, jy, l, k);
          int64_t j = idx3(n, i, jy, l);
          c2[j] += -I * k[a] * c[j];
        }
  }
  inv3_real(n, s, c2, out);
}

/* out = (D^T D)^+ g: divide the spectrum by |k_odd|^2 (0 where that is 0). */
static void aq_precond(int n, double s, const double* g, double* out, cplx* c) {
  int64_t tot = (int64_t)n * n * n;
  for (int64_t j = 0; j < tot; j++) c[j] = g[j];
  fwd3(n, s, c);
#pragma omp parallel for
  for (int l = 0; l < n; l++)
    for (int jy = 0; jy < n; jy++)
      for (int i = 0; i < n; i++) {
        double k[3];
        kvec_odd(n, s, i, jy, l, k);
        double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        int64_t j = idx3(n, i, jy, l);
        c[j] = kk > 0 ? c[j] / kk : 0;
      }
  inv3_real(n, s, c, out);
}

/* Compensated (Neumaier) summation: the energy differences the line search
 * compares shrink with the square of the gradient, far below the rounding
 * error of a plain sum over n^3 terms. */
typedef struct {
  double s, c;
} aq_sum;
static inline void aq_add(aq_sum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}

/* Sum of a[j] b[j] over m = n^3 terms: compensated partial sums per plane
 * (in parallel), combined in plane order, so that the result does not depend
 * on the number of threads. */
static double aq_dot(int64_t m, const double* a, const double* b) {
  int64_t nz = 1;
  while (nz * nz * nz < m) nz++;
  int64_t per = m / nz;
  double* part = (double*)malloc(sizeof(double) * (size_t)nz);
#pragma omp parallel for
  for (int64_t z = 0; z < nz; z++) {
    aq_sum t = {0, 0};
    for (int64_t j = z * per; j < (z + 1) * per; j++) aq_add(&t, a[j] * b[j]);
    part[z] = t.s + t.c;
  }
  aq_sum t = {0, 0};
  for (int64_t z = 0; z < nz; z++) aq_add(&t, part[z]);
  free(part);
  return t.s + t.c;
}

/* E(phi) and its gradient. u, w: 3-plane scratch. */
static double aq_energy(int n, double s, double a0, int kind, const double* gN, const double* phi, double* grad,
                        double* u, double* w, cplx* c, cplx* c2) {
  int64_t tot = (int64_t)n * n * n;
  aq_grad(n, s, phi, u, c, c2);
  const int64_t plane = (int64_t)n * n;
  double* part = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp parallel for
  for (int z = 0; z < n; z++) {
    aq_sum e = {0, 0};
    for (int64_t j = z * plane; j < (z + 1) * plane; j++) {
      double um = 0;
      for (int a = 0; a < 3; a++) {
        um += u[a * tot + j] * u[a * tot + j];
        aq_add(&e, gN[a * tot + j] * u[a * tot + j]);
      }
      um = sqrt(um);
      aq_add(&e, a0 * a0 * psi_mu(kind, um / a0));
      double m = ora_mu(kind, um / a0);
      for (int a = 0; a < 3; a++) w[a * tot + j] = m * u[a * tot + j] + gN[a * tot + j];
    }
    part[z] = e.s + e.c;
  }
  aq_sum e = {0, 0};
  for (int z = 0; z < n; z++) aq_add(&e, part[z]);
  free(part);
  aq_gradT(n, s, w, grad, c, c2);
  return e.s + e.c;
}

#define AQ_M 8
int ora_aqual_solve(int n, double s, double G, double a0, int mu_kind, const double* rho, const double* phi0,
                    double tol, int max_iter, double* phi_out, double* acc_out, double* info) {
  int64_t tot = (int64_t)n * n * n;
  double* gN = (double*)malloc(sizeof(double) * 3 * tot);
  double* u = (double*)malloc(sizeof(double) * 3 * tot);
  double* w = (double*)malloc(sizeof(double) * 3 * tot);
  double* x = (double*)malloc(sizeof(double) * tot);
  double* g = (double*)malloc(sizeof(double) * tot);
  double* xn = (double*)malloc(sizeof(double) * tot);
  double* gn = (double*)malloc(sizeof(double) * tot);
  double* q = (double*)malloc(sizeof(double) * tot);
  double* z = (double*)malloc(sizeof(double) * tot);
  double* S = (double*)malloc(sizeof(double) * AQ_M * tot);
  double* Y = (double*)malloc(sizeof(double) * AQ_M * tot);
  cplx* c = (cplx*)malloc(sizeof(cplx) * tot);
  cplx* c2 = (cplx*)malloc(sizeof(cplx) * tot);
  if (!gN || !u || !w || !x || !g || !xn || !gn || !q || !z || !S || !Y || !c || !c2) return ORA_ENOMEM;
  int rc = ora_solve(n, s, G, a0, mu_kind, 0, rho, NULL, 0, gN, NULL, NULL, NULL, NULL, NULL);
  if (rc != ORA_OK) return rc;
  /* scale of the gradient: |D^T g_N| */
  aq_gradT(n, s, gN, q, c, c2);
  double g0 = sqrt(aq_dot(tot, q, q));
  if (phi0) memcpy(x, phi0, sizeof(double) * tot);
  else memset(x, 0, sizeof(double) * tot);
  double e = aq_energy(n, s, a0, mu_kind, gN, x, g, u, w, c, c2);
  int evals = 1, it = 0, m = 0, head = 0;
  double rel = g0 > 0 ? sqrt(aq_dot(tot, g, g)) / g0 : 0.0;
  double rho_k[AQ_M], alpha[AQ_M];
  while (rel > tol && it < max_iter) {
    /* two-loop recursion: z = H g with H0 = gamma (D^T D)^+ */
    memcpy(q, g, sizeof(double) * tot);
    for (int t = 0; t < m; t++) {
      int b = (head - 1 - t + AQ_M) % AQ_M;
      alpha[b] = rho_k[b] * aq_dot(tot, S + b * tot, q);
#pragma omp parallel for
      for (int64_t j = 0; j < tot; j++) q[j] -= alpha[b] * Y[b * tot + j];
    }
    aq_precond(n, s, q, z, c);
    if (m > 0) {
      int b = (head - 1 + AQ_M) % AQ_M;
      aq_precond(n, s, Y + b * tot, xn, c);
      double gam = aq_dot(tot, S + b * tot, Y + b * tot) / aq_dot(tot, Y + b * tot, xn);
#pragma omp parallel for
      for (int64_t j = 0; j < tot; j++) z[j] *= gam;
    }
    for (int t = m - 1; t >= 0; t--) {
      int b = (head - 1 - t + AQ_M) % AQ_M;
      double beta = rho_k[b] * aq_dot(tot, Y + b * tot, z);
#pragma omp parallel for
      for (int64_t j = 0; j < tot; j++) z[j] += S[b * tot + j] * (alpha[b] - beta);
    }
    /* direction -z; backtracking until E falls by the Armijo fraction */
    double gd = -aq_dot(tot, g, z), step = 1.0, en = 0;
    int ok = 0;
    if (gd < 0) {
      for (int tries = 0; tries < 30; tries++, step *= 0.5) {
#pragma omp parallel for
        for (int64_t j = 0; j < tot; j++) xn[j] = x[j] - step * z[j];
        en = aq_energy(n, s, a0, mu_kind, gN, xn, gn, u, w, c, c2);
        evals++;
        if (en <= e + 1e-4 * step * gd) {
          ok = 1;
          break;
        }
      }
    }
    if (!ok) break; /* E can no longer be lowered at this precision */
    double sy = 0;
#pragma omp parallel for
    for (int64_t j = 0; j < tot; j++) {
      S[head * tot + j] = xn[j] - x[j];
      Y[head * tot + j] = gn[j] - g[j];
    }
    sy = aq_dot(tot, S + head * tot, Y + head * tot);
    if (sy > 0) {
      rho_k[head] = 1.0 / sy;
      head = (head + 1) % AQ_M;
      if (m < AQ_M) m++;
    }
    memcpy(x, xn, sizeof(double) * tot);
    memcpy(g, gn, sizeof(double) * tot);
    e = en;
    it++;
    rel = g0 > 0 ? sqrt(aq_dot(tot, g, g)) / g0 : 0.0;
  }
  if (phi_out) memcpy(phi_out, x, sizeof(double) * tot);
  if (acc_out) {
    fd_grad(n, s, x, acc_out);
    for (int64_t j = 0; j < 3 * tot; j++) acc_out[j] = -acc_out[j];
  }
  if (info) {
    info[0] = it;
    info[1] = rel;
    info[2] = evals;
  }
  free(gN); free(u); free(w); free(x); free(g); free(xn); free(gn); free(q); free(z); free(S); free(Y);
  free(c); free(c2);
  return ORA_OK;
}
