// passes.cuh -- the mesh passes of the field solve (Sect. 2.1 iteration,
// App. Flow steps 3-9), as templates over the FFT-domain side N.
//
// Data layout in HBM:
//  real planes     float [z][y][x], N^3 values (x fastest)
//  spectral planes float2 [z][y][kx], kx = 0..N/2 in rows of SP = N/2 + 2
//                  complex (16-byte aligned rows); y and z are either real
//                  coordinates or frequencies depending on the stage.
// A 3-D transform is an x-pass (R2C / C2R on contiguous lines), a y-pass and
// a z-pass (C2C on strided lines, tiles of P adjacent kx columns). The
// pointwise steps of the iteration (nu, mu, H = F - g_N) live inside x-passes;
// the spectral operators (Poisson, projections, gradient) inside z-passes,
// between the forward and the inverse z transform. Transforms are
// unnormalised; each z-pass multiplies by 1/N^3, the product of the s^3 and
// L^-3 of App. Fourier.
#pragma once
#include "fft.cuh"
#include "tma.cuh"

namespace passes {

constexpr int NT = 256;   // threads per CTA of the y- and z-passes
constexpr int NTX = 256;  // threads per CTA of the x-pass

template <int N>
struct XCfg {
  static constexpr int L = N >= 384 ? 8 : 16;  // lines per CTA
  static constexpr int LP = L + 1;             // padded line pitch in shared memory (bank spread)
  static constexpr int H = N / 2;              // complex FFT length of the real transform
  static constexpr int ROWS = H + 1;           // spectral positions 0..N/2
  static constexpr int SP = N / 2 + 2;
};

template <int N>
struct YZCfg {
  static constexpr int P = N >= 384 ? 8 : 16;    // kx columns per tile
  static constexpr int SP = N / 2 + 2;
  static constexpr int NX = N / 2 + 1;           // valid kx columns
  static constexpr int NBLK = (NX + P - 1) / P;  // tiles across kx
};

// x-pass modes
enum XMode {
  X_RHO = 0,       // int64 deposit -> FP32 density (exact rule), R2C
  X_NU_FIRST = 1,  // C2R g_N (store), F = g_N + H0, g_M = nu(F) F, R2C
  X_NU = 2,        // C2R H (optionally store, track dH), F = g_N + H, g_M = nu(F) F, R2C
  X_MU = 3,        // C2R g_M, F = mu(g_M) g_M, H = F - g_N, R2C
  X_INV = 4,       // C2R -> real planes
  X_FWD = 5,       // real planes -> R2C
  X_NU_REAL = 6,   // stored g_N (real) + H0, g_M = nu(F) F, R2C (reuses the last Newton solve)
  // incremental solve (Sect. 5.2 v): increments about a base state, nu and mu linearised
  X_DRHO = 7,      // two int64 deposits -> FP32 density increment (integer difference), base := new; R2C
  X_DNU_FIRST = 8, // C2R dg_N (store), dg_M = Jnu(g_N + H0) dg_N, R2C
  X_DNU = 9,       // C2R dH, dg_M = Jnu(g_N + H0) (dg_N + dH), R2C
  X_DMU = 10       // C2R dg_M, dH = Jmu(g_M0) dg_M - dg_N (optionally move the base on), R2C
};

// z-pass modes
enum ZMode {
  Z_NEWTON = 0,      // 1 -> 3 (+phi): g_N^ = i kappa 4 pi G A rho^
  Z_CURL = 1,        // 3 -> 3: curl-free projection
  Z_DIV = 2,         // 3 -> 3: divergence-free projection
  Z_FINAL = 3,       // 3 -> 3 (+phi) to out: a^ = -i kappa phi^, phi^ = i A k'.g^
  Z_SMOOTH = 5       // 3 -> 3: times the smoothing kernel spectrum
};

struct XArgs {
  float2* spec;          // spectral planes in/out (in place), component c at spec + c * pstride
  int64_t pstride;       // spectral plane stride (complex elements)
  float* real_out;       // X_INV destinations: compact real planes, stride N^3
  float* real_out2;      // X_INV second destinations (may be null)
  const float* real_in;  // X_FWD sources, stride N^3
  const float* gN;       // 3 real planes
  float* gN_out;         // X_NU_FIRST: where g_N is written
  const float* H0;       // X_NU_FIRST: warm H (3 real planes) or null
  float* Hs_out;         // X_NU: store H (3 real planes) or null
  uint64_t* dep;         // X_RHO: accumulator
  float* rho_out;        // X_RHO: density plane (may be null)
  double rho_scale;      // X_RHO: 2^-Kacc / s^3
  int rho_pow2;          // X_RHO, X_DRHO: 1 when rho_scale is exactly 2^rho_exp2 (the integer path of rho_rule)
  int rho_exp2;
  int ext_axis1;         // X_RHO, X_FWD of a density: 1 + axis of the external-field dipole layer, 0 none
  float ext_rho;         // its density: +ext_rho on the last plane along that axis, -ext_rho on the first
  double* red;           // dH reduction slots (2 doubles) or null
  float* gM_out;         // X_MU: store the curl-free g_M it reads (the mu base of an incremental solve)
  uint64_t* dep0;        // X_DRHO: base accumulator (read, then overwritten by dep)
  const float* dgN;      // X_DNU, X_DMU: density increment's Newton field (3 real planes)
  float* gM0;            // X_DMU: base g_M (3 real planes; += dg_M when base_update)
  float* gN_upd;         // X_DMU with base_update: g_N += dg_N
  int base_update;       // X_DMU: move the base on (last iteration)
  int accumulate;        // X_INV: real_out += the transformed planes
  const float2* tw;      // twiddles, N entries
  uint32_t* status;
  int mu_kind;
  float a0;
  float inv_a0, sqrt_a0;  // 1 / a0 and sqrt(a0) (the deep-MOND steps)
  int ncomp;
};

struct ZArgs {
  float2* in;       // input planes, component c at in + c * pstride
  float2* out;      // Z_NEWTON / Z_FINAL outputs (same stride)
  int64_t pstride;
  int nout;         // 3 or 4 (4: also phi)
  const float* kv;  // k values per index (N)
  const float* kp;  // kappa = sin(k s)/s per index (N)
  const float2* tw;
  const float* khat;  // smoothing kernel spectrum [z][y][kx] (N * N * (N/2+1))
  float norm;         // 1/N^3
  float coef;         // Z_NEWTON: 4 pi G
};

struct YArgs {
  float2* spec;  // component c at spec + c * pstride
  int64_t pstride;
  const float2* tw;
};

// ---------------------------------------------------------------------------
// Interpolation functions (Eq. mu and the pair relation of Sect. 2.1), FP32.
// nu_factor returns |g_M| / |F| for |F| = Fm; mu_factor returns |F| / |g_M|.
// Both are 0 at zero field.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float nu_factor(int kind, float Fm, float a0) {
  if (!(Fm > 0.0f)) return 0.0f;
  float y = Fm / a0;
  switch (kind) {
    case 0: return sqrtf(a0 / Fm);                       // deep: 1/sqrt(y)
    case 1: return 0.5f + sqrtf(0.25f + a0 / Fm);        // simple
    case 2:                                              // standard
      if (y > 1.0f) return sqrtf(0.5f + 0.5f * sqrtf(1.0f + 4.0f / (y * y)));
      return sqrtf((y + sqrtf(y * y + 4.0f)) / (2.0f * y));
    default: return 1.0f;
  }
}
__device__ __forceinline__ float mu_factor(int kind, float gm, float a0) {
  float x = gm / a0;
  switch (kind) {
    case 0: return x;                                    // deep
    case 1: return x / (1.0f + x);                       // simple
    case 2:                                              // standard
      if (x > 1.0f) return 1.0f / sqrtf(1.0f + 1.0f / (x * x));
      return x / sqrtf(1.0f + x * x);
    default: return 1.0f;
  }
}

// y nu'(y) at y = Fm/a0 given nu = nu_factor(kind, Fm, a0) > 0, and x mu'(x)
// at x = gm/a0 given mu = mu_factor(kind, gm, a0) (the derivatives of the
// functions above, for the linearised steps of Sect. 5.2 v).
__device__ __forceinline__ float ynu_prime(int kind, float Fm, float a0, float nu) {
  switch (kind) {
    case 0: return -0.5f * nu;                                    // deep: -1/(2 sqrt y)
    case 1: return -0.5f * a0 / (Fm * (nu - 0.5f));               // simple: -1/(2 y sqrt(1/4 + 1/y))
    case 2: {                                                     // standard: -1/(nu y sqrt(y^2 + 4))
      float y = Fm / a0;
      return -1.0f / (nu * y * sqrtf(y * y + 4.0f));
    }
    default: return 0.0f;
  }
}
__device__ __forceinline__ float xmu_prime(int kind, float gm, float a0, float mu) {
  float x = gm / a0;
  switch (kind) {
    case 0: return x;                                             // deep
    case 1: return x / ((1.0f + x) * (1.0f + x));                 // simple
    case 2: {                                                     // standard: x/(1+x^2)^{3/2} = mu/(1+x^2)
      float r = x > 1.0f ? __frcp_rn(x * x) : 1.0f;
      return x > 1.0f ? mu * r / (1.0f + r) : mu / (1.0f + x * x);
    }
    default: return 0.0f;
  }
}

// Linearised step about the point P (3 components) applied to d, in place:
// d <- f(p) d + p f'(p) (u.d) u, p = |P|/a0, u = P/|P|, f = nu (MU = false)
// or mu (MU = true). The identity for the Newtonian kind; 0 where P = 0.
template <bool MU>
__device__ __forceinline__ void linearised(int kind, float a0, const float* P, float* d) {
  if (kind == 3) return;
  const float m = sqrtf(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
  if (!(m > 0.0f)) {
    d[0] = d[1] = d[2] = 0.0f;
    return;
  }
  float f, fp;
  if constexpr (MU) {
    f = mu_factor(kind, m, a0);
    fp = xmu_prime(kind, m, a0, f);
  } else {
    f = nu_factor(kind, m, a0);
    fp = ynu_prime(kind, m, a0, f);
  }
  const float im = __frcp_rn(m);
  const float ud = (P[0] * d[0] + P[1] * d[1] + P[2] * d[2]) * im;
  const float c = fp * ud * im;
  for (int a = 0; a < 3; a++) d[a] = f * d[a] + c * P[a];
}

// The deposit's density rule, float(double(v) * scale) for an int64 total v.
// When scale is an exact power of two, 2^e, the product only shifts the
// exponent, and the two roundings of the rule are done on the integer
// instead (the int64 -> double rounding to 53 bits, then the double -> float
// rounding to 24 bits, each to nearest, ties to even); this GPU's FP64 rate
// is low. Results outside the range of normal floats take the FP64 route.
__device__ __forceinline__ uint64_t round_to_bits(uint64_t a, int bits) {
  const int len = 64 - __clzll((long long)a);
  if (len <= bits) return a;
  const int d = len - bits;
  const uint64_t low = a & ((1ull << d) - 1ull), half = 1ull << (d - 1);
  uint64_t m = a >> d;
  if (low > half || (low == half && (m & 1ull))) m += 1ull;
  return m << d;  // exact (a < 2^63)
}
__device__ __forceinline__ float rho_rule(long long v, double scale, int pow2, int e) {
  if (pow2 && v != 0) {
    const uint64_t mag = v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;  // |v|, also for the most negative v
    const uint64_t a = round_to_bits(round_to_bits(mag, 53), 24);
    const int len = 64 - __clzll((long long)a);
    const int ex = len - 1 + e;  // unbiased exponent of the result
    if (ex >= -126 && ex <= 127) {
      const uint32_t mant = (uint32_t)((len > 24 ? a >> (len - 24) : a << (24 - len)) & 0x7FFFFFull);
      const uint32_t bits = ((uint32_t)(v < 0) << 31) | ((uint32_t)(ex + 127) << 23) | mant;
      return __uint_as_float(bits);
    }
  }
  return __double2float_rn(__dmul_rn(__ll2double_rn(v), scale));
}

// ---------------------------------------------------------------------------
// x-pass
// ---------------------------------------------------------------------------
// Dipole layer of the external field (Sect. 5.3) at samples x, x + 1 of line
// `line` (= z N + y): +ext_rho on the last plane along axis ext_axis1 - 1,
// -ext_rho on the first.
template <int N>
__device__ __forceinline__ float2 dipole2(const XArgs& a, int64_t line, int x) {
  int v0, v1;
  if (a.ext_axis1 == 1) {
    v0 = x;
    v1 = x + 1;
  } else {
    v0 = v1 = a.ext_axis1 == 2 ? (int)(line % N) : (int)(line / N);
  }
  const float e0 = v0 == N - 1 ? a.ext_rho : (v0 == 0 ? -a.ext_rho : 0.f);
  const float e1 = v1 == N - 1 ? a.ext_rho : (v1 == 0 ? -a.ext_rho : 0.f);
  return make_float2(e0, e1);
}

// Issue the asynchronous copies of one component's spectral tile into the
// transposed shared layout [kk][line]; they complete at tma::async_wait_all,
// so the tiles of all components are in flight together.
template <int N>
__device__ __forceinline__ void x_load_spec(float2* sm, const float2* __restrict__ g, int64_t line0, int tid) {
  using C = XCfg<N>;
  constexpr int SPL = C::H + 1;  // complex values of a line that are used (kx = 0..N/2)
  const float2* src = g + line0 * C::SP;
  const uint64_t pol = tma::policy_evict_first();  // read once: keep L2 for the prefetched planes
  // a warp per line, lanes along it (no division of the element index)
  const int warp = tid >> 5, lane = tid & 31;
  for (int l = warp; l < C::L; l += NTX / 32) {
    const float2* s = src + (int64_t)l * C::SP;
    for (int kk = lane; kk < SPL; kk += 32) tma::async_copy8_stream(sm + kk * C::LP + l, s + kk, pol);
  }
}

template <int N>
__device__ __forceinline__ void x_store_spec(const float2* sm, float2* __restrict__ g, int64_t line0, int tid) {
  using C = XCfg<N>;
  constexpr int Q = C::SP / 2;
  float4* dst = reinterpret_cast<float4*>(g + line0 * C::SP);
  // a warp per line, lanes along it (no division of the element index)
  const int warp = tid >> 5, lane = tid & 31;
  for (int l = warp; l < C::L; l += NTX / 32) {
    for (int qq = lane; qq < Q; qq += 32) {
      const int kk = 2 * qq;
      float2 a = sm[kk * C::LP + l];
      float2 b = (kk + 1 <= C::H) ? sm[(kk + 1) * C::LP + l] : make_float2(0.f, 0.f);
      __stcs(dst + l * Q + qq, make_float4(a.x, a.y, b.x, b.y));
    }
  }
}

// Half-spectrum X[0..N/2] -> Y[0..N/2-1] = 2E + 2iO (see x_post for E, O);
// a length-N/2 inverse transform of Y then yields x[2j] + i x[2j+1].
// The imaginary parts of X[0] and X[N/2] are dropped (real part of the inverse).
template <int N>
__device__ __forceinline__ void x_pre_c2r(float2* sm0, int nc, const float2* tw, int tid) {
  using C = XCfg<N>;
  constexpr int NP = N / 4 + 1;  // pairs (k, N/2 - k), k = 0..N/4
  constexpr int TILE = C::ROWS * C::LP;
  constexpr int KS = NTX / C::L;  // a thread keeps its line l and takes every KS-th pair
  static_assert(NTX % C::L == 0, "lines divide the threads");
  const int l = tid % C::L;
  for (int c = 0; c < nc; c++) {
    float2* sm = sm0 + c * TILE;  // component tile
#pragma unroll
    for (int k = tid / C::L; k < NP; k += KS) {
      if (k == 0) {
        float x0 = sm[0 * C::LP + l].x, xn = sm[C::H * C::LP + l].x;
        sm[0 * C::LP + l] = make_float2(x0 + xn, x0 - xn);
      } else {
        int k2 = C::H - k;
        float2 a = sm[k * C::LP + l], b = sm[k2 * C::LP + l];
        float2 w = tw[k];  // e^{+2 pi i k / N}
        float2 ya = cadd(cadd(a, cconj(b)), cmul_i<1>(cmul(w, csub(a, cconj(b)))));
        if (k2 != k) {
          float2 w2 = make_float2(-w.x, w.y);  // e^{+2 pi i (N/2-k)/N} = -conj(w)
          float2 yb = cadd(cadd(b, cconj(a)), cmul_i<1>(cmul(w2, csub(b, cconj(a)))));
          sm[k2 * C::LP + l] = yb;
        }
        sm[k * C::LP + l] = ya;
      }
    }
  }
  __syncthreads();
}

// Z = DFT_{N/2}(x[2j] + i x[2j+1]) -> X[k] = E[k] + W^k O[k], k = 0..N/2,
// E = (Z[k] + conj Z[N/2-k])/2, O = (Z[k] - conj Z[N/2-k])/(2i), W = e^{-2 pi i/N}.
template <int N>
__device__ __forceinline__ void x_post_r2c(float2* sm0, int nc, const float2* tw, int tid) {
  using C = XCfg<N>;
  constexpr int NP = N / 4 + 1;
  constexpr int TILE = C::ROWS * C::LP;
  constexpr int KS = NTX / C::L;  // a thread keeps its line l and takes every KS-th pair
  const int l = tid % C::L;
  for (int c = 0; c < nc; c++) {
    float2* sm = sm0 + c * TILE;  // component tile
#pragma unroll
    for (int k = tid / C::L; k < NP; k += KS) {
      if (k == 0) {
        float2 z = sm[0 * C::LP + l];
        sm[0 * C::LP + l] = make_float2(z.x + z.y, 0.f);
        sm[C::H * C::LP + l] = make_float2(z.x - z.y, 0.f);
      } else {
        int k2 = C::H - k;
        float2 a = sm[k * C::LP + l], b = sm[k2 * C::LP + l];
        float2 w = tw[k];               // (cos, sin)(2 pi k/N)
        float2 wc = cconj(w);           // e^{-2 pi i k/N}
        float2 e = cscale(cadd(a, cconj(b)), 0.5f);
        float2 d = cscale(csub(a, cconj(b)), 0.5f);
        float2 xa = csub(e, cmul_i<1>(cmul(wc, d)));  // E - i W^k (a - conj b)/2
        if (k2 != k) {
          float2 e2 = cscale(cadd(b, cconj(a)), 0.5f);
          float2 d2 = cscale(csub(b, cconj(a)), 0.5f);
          float2 xb = cadd(e2, cmul_i<1>(cmul(w, d2)));  // X[N/2-k]
          sm[k2 * C::LP + l] = xb;
        }
        sm[k * C::LP + l] = xa;
      }
    }
  }
  __syncthreads();
}

// The half-length complex transforms of all nc component tiles of an x-pass
// tile in one pass of barriers.
template <int N, int DIR>
__device__ __forceinline__ void xfft(float2* buf, int nc, const float2* tw, int tid) {
  using C = XCfg<N>;
  constexpr int TILE = C::ROWS * C::LP;
  // two component tiles per pass of barriers (one radix-16 butterfly per thread), then the rest
  int c = 0;
  for (; c + 2 <= nc; c += 2) fftk::fft_c<C::H, DIR, C::L, 2, NTX>(buf + c * TILE, C::LP, 1, TILE, tw, 2, tid);
  if (c < nc) fftk::fft_c<C::H, DIR, C::L, 1, NTX>(buf + c * TILE, C::LP, 1, TILE, tw, 2, tid);
}

template <int N, int MODE>
__global__ void __launch_bounds__(NTX) k_xpass(XArgs a, int64_t nlines) {
  using C = XCfg<N>;
  extern __shared__ float2 smem[];
  float2* tw = smem;                       // N twiddles
  float2* buf = smem + N;                  // ncomp tiles of ROWS x LP
  constexpr int TILE = C::ROWS * C::LP;
  const int tid = threadIdx.x;
  const int64_t line0 = (int64_t)blockIdx.x * C::L;
  for (int i = tid; i < N; i += NTX) tw[i] = a.tw[i];
  const int nc = (MODE == X_RHO || MODE == X_DRHO) ? 1 : a.ncomp;

  constexpr bool INC = (MODE == X_DNU_FIRST || MODE == X_DNU || MODE == X_DMU);  // incremental, 3 components
  constexpr bool INV = (MODE == X_NU_FIRST || MODE == X_NU || MODE == X_MU || MODE == X_INV || INC);
  constexpr bool FWD = (MODE == X_RHO || MODE == X_NU_FIRST || MODE == X_NU || MODE == X_MU || MODE == X_FWD ||
                        MODE == X_NU_REAL || MODE == X_DRHO || INC);

  if (tid == 0) {
    // the real-space planes the pointwise stage reads, brought into L2 while
    // the spectral tile is loaded and transformed (L lines: contiguous)
    const uint32_t rb = (uint32_t)(C::L * N * sizeof(float));
    const int64_t r0 = line0 * N;
    for (int c = 0; c < 3; c++) {
      const int64_t o = (int64_t)c * N * N * N + r0;
      if constexpr (MODE == X_NU || MODE == X_MU || MODE == X_NU_REAL) tma::prefetch_l2(a.gN + o, rb);
      if constexpr (MODE == X_NU_FIRST || MODE == X_NU_REAL)
        if (a.H0) tma::prefetch_l2(a.H0 + o, rb);
      if constexpr (MODE == X_NU)
        if (a.Hs_out && a.red) tma::prefetch_l2(a.Hs_out + o, rb);
      if constexpr (MODE == X_DNU_FIRST || MODE == X_DNU) {
        tma::prefetch_l2(a.gN + o, rb);
        tma::prefetch_l2(a.H0 + o, rb);
      }
      if constexpr (MODE == X_DNU || MODE == X_DMU) tma::prefetch_l2(a.dgN + o, rb);
      if constexpr (MODE == X_DMU) tma::prefetch_l2(a.gM0 + o, rb);
    }
  }
  if constexpr (INV) {
    for (int c = 0; c < nc; c++) x_load_spec<N>(buf + c * TILE, a.spec + c * a.pstride, line0, tid);
    tma::async_wait_all();
    __syncthreads();
    x_pre_c2r<N>(buf, nc, tw, tid);
    xfft<N, +1>(buf, nc, tw, tid);
  }

  // Pointwise stage on real samples: point (j, l) holds x[2j], x[2j+1] of line l.
  const int64_t rbase = line0 * N;  // real index of the first sample of the tile
  float sq_dh = 0.f, sq_gn = 0.f;
  bool bad = false;
  if constexpr (MODE == X_RHO) {
    // the density: all of a thread's accumulator loads in flight at once, then the rule
    constexpr int PER = (C::L * C::H + NTX - 1) / NTX;
    ulonglong2 u[PER];
#pragma unroll
    for (int k = 0; k < PER; k++) {
      const int i = tid + k * NTX, j = i % C::H, l = i / C::H;
      if (i < C::L * C::H) u[k] = __ldcs(reinterpret_cast<const ulonglong2*>(a.dep + rbase + (int64_t)l * N + 2 * j));
    }
#pragma unroll
    for (int k = 0; k < PER; k++) {
      const int i = tid + k * NTX, j = i % C::H, l = i / C::H;
      if (i >= C::L * C::H) break;
      const int64_t ri = rbase + (int64_t)l * N + 2 * j;
      float r0 = rho_rule((long long)u[k].x, a.rho_scale, a.rho_pow2, a.rho_exp2);
      float r1 = rho_rule((long long)u[k].y, a.rho_scale, a.rho_pow2, a.rho_exp2);
      if (a.rho_out) *reinterpret_cast<float2*>(a.rho_out + ri) = make_float2(r0, r1);
      if (a.ext_axis1) {
        const float2 e = dipole2<N>(a, line0 + l, 2 * j);
        r0 += e.x;
        r1 += e.y;
      }
      buf[j * C::LP + l] = make_float2(r0, r1);
    }
  }
  for (int i = tid; MODE != X_RHO && i < C::L * C::H; i += NTX) {
    int j = i % C::H, l = i / C::H;
    int64_t ri = rbase + (int64_t)l * N + 2 * j;
    float2* const p0 = buf + j * C::LP + l;  // component c at p0 + c * TILE
    if constexpr (MODE == X_DRHO) {
      // increment of two deposits: the int64 difference first (exact), then the
      // density rule; the new deposit becomes the base
      ulonglong2 u = *reinterpret_cast<const ulonglong2*>(a.dep + ri);
      ulonglong2* bp = reinterpret_cast<ulonglong2*>(a.dep0 + ri);
      ulonglong2 u0 = *bp;
      *bp = u;
      float r0 = rho_rule((long long)(u.x - u0.x), a.rho_scale, a.rho_pow2, a.rho_exp2);
      float r1 = rho_rule((long long)(u.y - u0.y), a.rho_scale, a.rho_pow2, a.rho_exp2);
      *p0 = make_float2(r0, r1);
    } else if constexpr (INC) {
      const int64_t P3 = (int64_t)N * N * N;
      float v[3][2], dg[3][2], bs[3][2];
      for (int c = 0; c < 3; c++) {
        float2 t = p0[c * TILE];
        v[c][0] = t.x;
        v[c][1] = t.y;
      }
      if constexpr (MODE == X_DNU_FIRST) {
        // input is dg_N: store it; dF = dg_N
        for (int c = 0; c < 3; c++)
          *reinterpret_cast<float2*>(a.gN_out + c * P3 + ri) = make_float2(v[c][0], v[c][1]);
      } else {
        for (int c = 0; c < 3; c++) {
          float2 t = *reinterpret_cast<const float2*>(a.dgN + c * P3 + ri);
          dg[c][0] = t.x;
          dg[c][1] = t.y;
        }
      }
      if constexpr (MODE == X_DNU)
        for (int c = 0; c < 3; c++) {  // dF = dg_N + dH
          v[c][0] += dg[c][0];
          v[c][1] += dg[c][1];
        }
      // the linearisation point: F0 = g_N + H0 (nu steps) or g_M0 (mu step)
      for (int c = 0; c < 3; c++) {
        float2 t;
        if constexpr (MODE == X_DMU) {
          t = *reinterpret_cast<const float2*>(a.gM0 + c * P3 + ri);
        } else {
          t = *reinterpret_cast<const float2*>(a.gN + c * P3 + ri);
          float2 h0 = *reinterpret_cast<const float2*>(a.H0 + c * P3 + ri);
          t.x += h0.x;
          t.y += h0.y;
        }
        bs[c][0] = t.x;
        bs[c][1] = t.y;
      }
      if constexpr (MODE == X_DMU) {
        if (a.base_update) {
          // g_M0 += dg_M, g_N += dg_N: the base moves on to the new state
          for (int c = 0; c < 3; c++) {
            *reinterpret_cast<float2*>(a.gM0 + c * P3 + ri) =
                make_float2(bs[c][0] + v[c][0], bs[c][1] + v[c][1]);
            float* gp = a.gN_upd + c * P3 + ri;
            float2 g = *reinterpret_cast<const float2*>(gp);
            *reinterpret_cast<float2*>(gp) = make_float2(g.x + dg[c][0], g.y + dg[c][1]);
          }
        }
      }
      for (int e = 0; e < 2; e++) {
        float P[3] = {bs[0][e], bs[1][e], bs[2][e]};
        float d[3] = {v[0][e], v[1][e], v[2][e]};
        linearised<MODE == X_DMU>(a.mu_kind, a.a0, P, d);
        for (int c = 0; c < 3; c++) {
          float o = d[c];
          if constexpr (MODE == X_DMU) o -= dg[c][e];  // dH = dF - dg_N
          bad |= !isfinite(o);
          v[c][e] = o;
        }
      }
      for (int c = 0; c < 3; c++) p0[c * TILE] = make_float2(v[c][0], v[c][1]);
    } else if constexpr (MODE == X_FWD) {
      for (int c = 0; c < nc; c++) p0[c * TILE] = *reinterpret_cast<const float2*>(a.real_in + (int64_t)c * N * N * N + ri);
      if (a.ext_axis1) {
        const float2 e = dipole2<N>(a, line0 + l, 2 * j);
        p0[0].x += e.x;
        p0[0].y += e.y;
      }
    } else if constexpr (MODE == X_INV) {
      for (int c = 0; c < nc; c++) {
        float2 v = p0[c * TILE];
        bad |= !(isfinite(v.x) && isfinite(v.y));
        float2* dst = reinterpret_cast<float2*>(a.real_out + (int64_t)c * N * N * N + ri);
        if (a.accumulate) {
          const float2 o = *dst;
          v.x += o.x;
          v.y += o.y;
        }
        *dst = v;
        if (a.real_out2) *reinterpret_cast<float2*>(a.real_out2 + (int64_t)c * N * N * N + ri) = v;
      }
    } else {
      // three components, two samples each
      float v[3][2], gn[3][2];
      if constexpr (MODE != X_NU_REAL) {
        for (int c = 0; c < 3; c++) {
          float2 t = p0[c * TILE];
          v[c][0] = t.x;
          v[c][1] = t.y;
        }
      }
      if constexpr (MODE == X_NU_REAL) {
        // F = g_N + H0 from the stored Newton field
        for (int c = 0; c < 3; c++) {
          float2 t = *reinterpret_cast<const float2*>(a.gN + (int64_t)c * N * N * N + ri);
          float2 h0 = a.H0 ? *reinterpret_cast<const float2*>(a.H0 + (int64_t)c * N * N * N + ri)
                           : make_float2(0.f, 0.f);
          gn[c][0] = t.x;
          gn[c][1] = t.y;
          v[c][0] = t.x + h0.x;
          v[c][1] = t.y + h0.y;
        }
      } else if constexpr (MODE == X_NU_FIRST) {
        // input is g_N; store it; F = g_N + H0
        for (int c = 0; c < 3; c++) {
          *reinterpret_cast<float2*>(a.gN_out + (int64_t)c * N * N * N + ri) = make_float2(v[c][0], v[c][1]);
          gn[c][0] = v[c][0];
          gn[c][1] = v[c][1];
          float2 h0 = a.H0 ? *reinterpret_cast<const float2*>(a.H0 + (int64_t)c * N * N * N + ri)
                           : make_float2(0.f, 0.f);
          v[c][0] += h0.x;
          v[c][1] += h0.y;
        }
      } else {
        for (int c = 0; c < 3; c++) {
          float2 t = *reinterpret_cast<const float2*>(a.gN + (int64_t)c * N * N * N + ri);
          gn[c][0] = t.x;
          gn[c][1] = t.y;
        }
      }
      if constexpr (MODE == X_MU) {
        if (a.gM_out)
          for (int c = 0; c < 3; c++)
            *reinterpret_cast<float2*>(a.gM_out + (int64_t)c * N * N * N + ri) = make_float2(v[c][0], v[c][1]);
      }
      if constexpr (MODE == X_NU) {
        // input is H after the divergence-free projection
        if (a.Hs_out) {
          for (int c = 0; c < 3; c++) {
            float* hp = a.Hs_out + (int64_t)c * N * N * N + ri;
            if (a.red) {
              float2 old = *reinterpret_cast<const float2*>(hp);
              float d0 = v[c][0] - old.x, d1 = v[c][1] - old.y;
              sq_dh += d0 * d0 + d1 * d1;
              sq_gn += gn[c][0] * gn[c][0] + gn[c][1] * gn[c][1];
            }
            *reinterpret_cast<float2*>(hp) = make_float2(v[c][0], v[c][1]);
          }
        }
        for (int c = 0; c < 3; c++) {
          v[c][0] += gn[c][0];
          v[c][1] += gn[c][1];
        }
      }
      for (int e = 0; e < 2; e++) {
        float m2 = v[0][e] * v[0][e] + v[1][e] * v[1][e] + v[2][e] * v[2][e];
        float f;
        if (a.mu_kind == 0) {
          // deep MOND, from the hardware reciprocal square root (a few ulp, no
          // IEEE divide or square root): nu = sqrt(a0 / |F|) = sqrt(a0) (m2)^-1/4,
          // mu |g| / a0 with |g| = m2 / sqrt(m2); 0 at zero field
          const float r = m2 > 0.f ? rsqrtf(m2) : 0.f;  // 1 / |v|
          if constexpr (MODE == X_MU) f = m2 * r * a.inv_a0;
          else f = a.sqrt_a0 * (r * rsqrtf(r > 0.f ? r : 1.f)) * (r > 0.f ? 1.f : 0.f);
        } else {
          const float mag = sqrtf(m2);
          if constexpr (MODE == X_MU) f = mu_factor(a.mu_kind, mag, a.a0);
          else f = nu_factor(a.mu_kind, mag, a.a0);
        }
        for (int c = 0; c < 3; c++) {
          float o = f * v[c][e];
          if constexpr (MODE == X_MU) o -= gn[c][e];  // H = F - g_N
          v[c][e] = o;
        }
        bad |= !isfinite(m2);
      }
      for (int c = 0; c < 3; c++) p0[c * TILE] = make_float2(v[c][0], v[c][1]);
    }
  }
  if (bad) set_status(a.status, ST_NAN);
  if (MODE == X_NU && a.red && a.Hs_out) {
    // per-CTA partial sums of |dH|^2 and |g_N|^2
    for (int o = 16; o > 0; o >>= 1) {
      sq_dh += __shfl_xor_sync(0xffffffffu, sq_dh, o);
      sq_gn += __shfl_xor_sync(0xffffffffu, sq_gn, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(a.red, (double)sq_dh);
      atomicAdd(a.red + 1, (double)sq_gn);
    }
  }

  if constexpr (FWD) {
    __syncthreads();
    xfft<N, -1>(buf, nc, tw, tid);
    x_post_r2c<N>(buf, nc, tw, tid);
    for (int c = 0; c < nc; c++) x_store_spec<N>(buf + c * TILE, a.spec + c * a.pstride, line0, tid);
  }
}

// ---------------------------------------------------------------------------
// y-pass: C2C along y for one component per CTA, tile N (y) x P (kx).
// grid (NBLK, N (z), ncomp)
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void yz_load(float2* sm, const float2* __restrict__ g, int64_t row_stride, int col0,
                                        int tid) {
  using C = YZCfg<N>;
  constexpr int Q = C::P / 2;  // float4 per row
  int ncol = C::SP - col0;     // columns remaining in the row (includes the pad column)
  int q_valid = ncol >= C::P ? Q : (ncol + 1) / 2;
  for (int i = tid; i < N * Q; i += NT) {
    int row = i / Q, q = i % Q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < q_valid) v = __ldcs(reinterpret_cast<const float4*>(g + row * row_stride + col0) + q);
    sm[row * C::P + 2 * q] = make_float2(v.x, v.y);
    sm[row * C::P + 2 * q + 1] = make_float2(v.z, v.w);
  }
}

template <int N>
__device__ __forceinline__ void yz_store(const float2* sm, float2* __restrict__ g, int64_t row_stride, int col0,
                                         int tid) {
  using C = YZCfg<N>;
  constexpr int Q = C::P / 2;
  int ncol = C::SP - col0;
  int q_valid = ncol >= C::P ? Q : (ncol + 1) / 2;
  for (int i = tid; i < N * Q; i += NT) {
    int row = i / Q, q = i % Q;
    if (q < q_valid) {
      float2 a = sm[row * C::P + 2 * q], b = sm[row * C::P + 2 * q + 1];
      __stcs(reinterpret_cast<float4*>(g + row * row_stride + col0) + q, make_float4(a.x, a.y, b.x, b.y));
    }
  }
}

template <int N, int DIR>
__global__ void __launch_bounds__(NT) k_ypass(YArgs a) {
  using C = YZCfg<N>;
  extern __shared__ float2 smem[];
  float2* tw = smem;
  float2* tile = smem + N;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += NT) tw[i] = a.tw[i];
  const int col0 = blockIdx.x * C::P;
  const int z = blockIdx.y;
  float2* base = a.spec + blockIdx.z * a.pstride + (int64_t)z * N * C::SP;
  yz_load<N>(tile, base, C::SP, col0, tid);
  __syncthreads();
  fftk::fft<N, DIR, C::P, NT>(tile, C::P, 1, tw, 1, tid);
  yz_store<N>(tile, base, C::SP, col0, tid);
}

// ---------------------------------------------------------------------------
// z-pass: forward z, spectral operator, inverse z. grid (NBLK, N (y)).
// ---------------------------------------------------------------------------
template <int N, int MODE>
__global__ void __launch_bounds__(NT) k_zpass(ZArgs a) {
  using C = YZCfg<N>;
  extern __shared__ float2 smem[];
  float2* tw = smem;
  float* kv = reinterpret_cast<float*>(smem + N);
  float* kp = kv + N;
  float2* tile = smem + 2 * N;  // tiles of N x P
  constexpr int T = N * C::P;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += NT) {
    tw[i] = a.tw[i];
    kv[i] = a.kv[i];
    kp[i] = a.kp[i];
  }
  const int col0 = blockIdx.x * C::P;
  const int y = blockIdx.y;
  const int64_t rs = (int64_t)N * C::SP;  // z row stride
  const int64_t off = (int64_t)y * C::SP;
  constexpr int NIN = (MODE == Z_NEWTON) ? 1 : 3;
  for (int c = 0; c < NIN; c++) yz_load<N>(tile + c * T, a.in + c * a.pstride + off, rs, col0, tid);
  __syncthreads();
  for (int c = 0; c < NIN; c++) fftk::fft<N, -1, C::P, NT>(tile + c * T, C::P, 1, tw, 1, tid);

  // spectral operator at (kx = col, ky = y, kz = row)
  const float ky = kv[y];
  const bool ny = (y == N / 2);
  const float kpy = kp[y];
  int nout_extra = 0;
  if constexpr (MODE == Z_NEWTON || MODE == Z_FINAL) nout_extra = a.nout;
  for (int i = tid; i < T; i += NT) {
    int row = i / C::P, cc = i % C::P;
    int col = col0 + cc;
    if (col > N / 2) continue;
    float kx = kv[col], kz = kv[row];
    bool nx = (col == N / 2), nz = (row == N / 2);
    float kk = kx * kx + ky * ky + kz * kz;
    float A = kk > 0.f ? __frcp_rn(kk) : 0.f;  // correctly rounded, as 1.0f / kk
    float kpx = kp[col], kpz = kp[row];
    if constexpr (MODE == Z_NEWTON) {
      float2 r = tile[i];
      float f = a.coef * A * a.norm;  // 4 pi G A / N^3
      float2 ir = cmul_i<1>(r);       // i rho^
      tile[i] = cscale(ir, f * kpx);
      tile[T + i] = cscale(ir, f * kpy);
      tile[2 * T + i] = cscale(ir, f * kpz);
      if (nout_extra == 4) tile[3 * T + i] = cscale(r, -f);  // phi_N^ = -4 pi G A rho^
    } else if constexpr (MODE == Z_SMOOTH) {
      int64_t kidx = ((int64_t)row * N + y) * (N / 2 + 1) + col;
      float f = a.khat[kidx] * a.norm;
      for (int c = 0; c < 3; c++) tile[c * T + i] = cscale(tile[c * T + i], f);
    } else {
      float2 g0 = tile[i], g1 = tile[T + i], g2 = tile[2 * T + i];
      float k3[3] = {kx, ky, kz};
      bool n3[3] = {nx, ny, nz};
      if constexpr (MODE == Z_FINAL) {
        // phi^ = i A sum_b k'_b g_b (k'_b = 0 on the Nyquist plane of axis b)
        float2 S = make_float2(0.f, 0.f);
        float2 gg[3] = {g0, g1, g2};
        for (int b = 0; b < 3; b++)
          if (!n3[b]) S = cadd(S, cscale(gg[b], k3[b]));
        float f = A * a.norm;
        float2 aS = cscale(S, f);
        // a^ = -i kappa phi^ = kappa A S, times the smoothing spectrum when
        // the mesh is to hold the node-smoothed field
        const float fk = a.khat ? a.khat[((int64_t)row * N + y) * (N / 2 + 1) + col] : 1.0f;
        const float2 aK = cscale(aS, fk);
        float2* dst = tile;
        dst[i] = cscale(aK, kpx);
        dst[T + i] = cscale(aK, kpy);
        dst[2 * T + i] = cscale(aK, kpz);
        if (nout_extra == 4) dst[3 * T + i] = cmul_i<1>(aS);
      }
      if constexpr (MODE == Z_CURL || MODE == Z_DIV) {
        // P_ab = k_a k_b A, off-diagonal terms dropped when exactly one of
        // a, b sits on its Nyquist plane (real part of the inverse transform)
        float2 gg[3] = {g0, g1, g2};
        float2 o[3];
        for (int aa = 0; aa < 3; aa++) {
          float2 t = make_float2(0.f, 0.f);
          for (int b = 0; b < 3; b++)
            if (aa == b || n3[aa] == n3[b]) t = cadd(t, cscale(gg[b], k3[aa] * k3[b] * A));
          o[aa] = (MODE == Z_DIV) ? csub(gg[aa], t) : t;
        }
        for (int c = 0; c < 3; c++) tile[c * T + i] = cscale(o[c], a.norm);
      }
    }
  }
  __syncthreads();
  int nfin = (MODE == Z_NEWTON || MODE == Z_FINAL) ? a.nout : 3;
  for (int c = 0; c < nfin; c++) fftk::fft<N, +1, C::P, NT>(tile + c * T, C::P, 1, tw, 1, tid);
  if constexpr (MODE == Z_NEWTON || MODE == Z_FINAL) {
    for (int c = 0; c < a.nout; c++) yz_store<N>(tile + c * T, a.out + c * a.pstride + off, rs, col0, tid);
  } else {
    for (int c = 0; c < 3; c++) yz_store<N>(tile + c * T, a.in + c * a.pstride + off, rs, col0, tid);
  }
}

}  // namespace passes

// ===========================================================================
// Pipelined y- and z-passes: persistent CTAs stream tiles through a two-stage
// shared-memory ring. One thread issues TMA tile loads (completion on an
// mbarrier) for tile i+1 and TMA stores of tile i-1 while all threads
// transform tile i, so HBM traffic overlaps the shared-memory FFT.
// ===========================================================================

namespace passes {

// Tile geometry of the pipelined passes: P columns per tile (y: PY, z: PZ),
// row boxes of at most 256 (the TMA box limit) dividing N.
constexpr int pipe_py(int n) { return n >= 384 ? 8 : 16; }
constexpr int pipe_pz(int n) { return n >= 256 ? 4 : (n >= 192 ? 8 : 16); }
constexpr int pipe_box(int n) { return n <= 256 ? n : (n % 256 == 0 ? 256 : 128); }

template <int N>
struct PipeCfg {
  static constexpr int PY = pipe_py(N);
  static constexpr int PZ = pipe_pz(N);
  static constexpr int BOX = pipe_box(N);
  static constexpr int NBOX = N / BOX;
  static constexpr int NX = N / 2 + 1;
  static constexpr int NBLKY = (NX + PY - 1) / PY;
  static constexpr int NBLKZ = (NX + PZ - 1) / PZ;
};

// Polls after which the wait for a tile whose load was never issued gives
// up (the fault-injection hook below).
constexpr uint32_t kLostLoadWaitLimit = 1024;

struct PipeYArgs {
  int ncomp;  // components to transform (tiles = NBLKY * N * ncomp)
  const float2* tw;
  uint32_t* status;
  // Fault injection for tests of the bounded waits: the load of this tile is
  // never issued, so its wait runs out (-1: none).
  int lost_tile = -1;
  int max_ctas = 0;  // cap on the persistent grid (0: as many as fit the GPU)
};

struct PipeZArgs {
  int nout;  // Z_NEWTON / Z_FINAL outputs (3 or 4)
  // mean of the last two iterations' potentials: 1 = this Z_CURL also writes
  // its A k'.g (the potential's spectrum over i, before the inverse z
  // transform) to the scalar slot of the final spectra; 2 = this Z_FINAL
  // reads it back and takes the mean with its own. Needs the scalar region.
  int mean;
  // 1: only the tiles holding kx = N/2 or ky = N/2 (the rest is the folded z-pass's)
  int nyq_only;
  int max_ctas;  // cap on the persistent grid (0: as many as fit the GPU)
  const float* kv;
  const float* kp;
  const float2* tw;
  const float* khat;
  float norm;
  float coef;
  uint32_t* status;
};

// Common ring driver. LoadF(tile, stage_ptr, bar) issues the loads of a tile
// and returns the bytes expected; ComputeF(tile, stage_ptr) transforms it in
// place; StoreF(tile, stage_ptr) issues its stores (called by thread 0 after
// the proxy fence). When a bounded wait gives up, the CTA waits (bounded, at
// the full limit) for the one load it has issued into the other stage, so that
// no copy into its shared memory is in flight when it leaves, and stops.
// lost_tile (tests only): that tile's load is not issued and its wait gives
// up after kLostLoadWaitLimit polls; every other wait keeps the full limit.
template <typename LoadF, typename ComputeF, typename StoreF>
__device__ __forceinline__ void pipe_run(int ntiles, float2* stage0, int stage_elems, uint64_t* bars, uint32_t* status,
                                         LoadF load, ComputeF compute, StoreF store, int lost_tile = -1) {
  const int tid = threadIdx.x;
  const int cnt = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (tid == 0) {
    tma::mbar_init(&bars[0], 1);
    tma::mbar_init(&bars[1], 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0 && cnt > 0 && (int)blockIdx.x != lost_tile) {
    const uint32_t bytes = load(blockIdx.x, stage0, &bars[0]);
    (void)bytes;
  }
  for (int i = 0; i < cnt; i++) {
    const int s = i & 1;
    float2* st = stage0 + s * stage_elems;
    const int tile = blockIdx.x + i * gridDim.x;
    if (tid == 0 && i + 1 < cnt) {
      tma::bulk_wait_read<0>();  // the other stage's store has finished reading it
      if (tile + (int)gridDim.x != lost_tile) load(tile + gridDim.x, stage0 + (s ^ 1) * stage_elems, &bars[s ^ 1]);
    }
    const bool ok = tma::mbar_wait(&bars[s], (uint32_t)((i >> 1) & 1), status,
                                   tile == lost_tile ? kLostLoadWaitLimit : tma::kWaitLimit);
    if (__syncthreads_or(!ok)) {
      // give up: wait (bounded) for the load already issued into the other stage
      if (tid == 0 && i + 1 < cnt) tma::mbar_wait(&bars[s ^ 1], (uint32_t)(((i + 1) >> 1) & 1), status);
      break;
    }
    compute(tile, st);
    tma::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      store(tile, st);
      tma::bulk_commit();
    }
  }
  if (tid == 0) tma::bulk_wait_all();
}

template <int N, int DIR>
__global__ void __launch_bounds__(NT) k_ypass_pipe(const __grid_constant__ tma::TensorMap map, PipeYArgs a) {
  using C = PipeCfg<N>;
  constexpr int P = C::PY;
  extern __shared__ __align__(128) float2 psm[];
  __shared__ __align__(8) uint64_t bars[2];
  float2* tw = psm;
  float2* stage0 = psm + N;  // N twiddles (16-byte multiple for N >= 2)
  constexpr int SE = N * P;  // elements per stage
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += NT) tw[i] = a.tw[i];
  const int ntiles = C::NBLKY * N * a.ncomp;
  // tile -> (column block, z, component); coordinates of the 3-D map
  // (x: floats of a row, y: row within the plane, z: component * N + plane z)
  auto coords = [&](int t, int& x, int& zz) {
    const int blk = t % C::NBLKY;
    const int rest = t / C::NBLKY;  // component * N + z
    x = blk * 2 * P;
    zz = rest;
  };
  auto load = [&](int t, float2* dst, uint64_t* bar) -> uint32_t {
    int x, zz;
    coords(t, x, zz);
    tma::mbar_expect_tx(bar, SE * 8);
    for (int b = 0; b < C::NBOX; b++) tma::load_3d(dst + b * C::BOX * P, &map, x, b * C::BOX, zz, bar);
    return SE * 8;
  };
  auto compute = [&](int, float2* st) { fftk::fft<N, DIR, P, NT>(st, P, 1, tw, 1, tid); };
  auto store = [&](int t, const float2* src) {
    int x, zz;
    coords(t, x, zz);
    for (int b = 0; b < C::NBOX; b++) tma::store_3d(&map, x, b * C::BOX, zz, src + b * C::BOX * P);
  };
  pipe_run(ntiles, stage0, SE, bars, a.status, load, compute, store, a.lost_tile);
}

// z-pass over the tile of (column block, y): forward z, the spectral
// operator, inverse z. Each stage holds a vector region [z row][3][column]
// (4-D maps with the component as a dimension, so one FFT call transforms the
// three components) and, for Z_NEWTON and Z_FINAL, a scalar region
// [z row][column] for rho^ (input) or phi^ (output, component 3 of A).
// threads per pipelined z-pass CTA: at N = 256, 192 = one radix-16 butterfly
// per thread for the 3 x 4 sequences of a tile (four CTAs per SM); 384 elsewhere.
template <int N, int MODE>
constexpr int zthreads() { return N == 256 ? 192 : 384; }

// SC: a separate scalar region per stage (needed only when phi is stored);
// without it the Newton pass lands its scalar input in the last third of the
// vector region and reads it into registers before the outputs overwrite it,
// so that every mode runs with three-component stages (two CTAs per SM).
template <int N, int MODE, bool SC, int NTZ = zthreads<N, MODE>()>
__global__ void __launch_bounds__(NTZ, 768 / NTZ) k_zpass_pipe(const __grid_constant__ tma::TensorMap in_map,
                                                   const __grid_constant__ tma::TensorMap out_map,
                                                   const __grid_constant__ tma::TensorMap phi_map, PipeZArgs a) {
  using C = PipeCfg<N>;
  constexpr int P = C::PZ;
  constexpr bool SCALAR = (MODE == Z_NEWTON || MODE == Z_FINAL);
  constexpr int VP = 3 * P;                     // vector row pitch
  constexpr int SE = N * VP + (SC ? N * P : 0);
  constexpr int SOFF = SC ? N * VP : 2 * N * P;  // scalar region inside a stage
  extern __shared__ __align__(128) float2 psm[];
  __shared__ __align__(8) uint64_t bars[2];
  float2* tw = psm;
  float* kv = reinterpret_cast<float*>(psm + N);
  float* kp = kv + N;
  float2* stage0 = psm + 2 * N;
  const bool phi = SC && SCALAR && a.nout > 3;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += NTZ) {
    tw[i] = a.tw[i];
    kv[i] = a.kv[i];
    kp[i] = a.kp[i];
  }
  const int ntiles = a.nyq_only ? C::NBLKZ + N - 1 : C::NBLKZ * N;
  // nyq_only: the row ky = N/2 of every block, then the block of kx = N/2 at every other row
  auto tile_at = [&](int t, int& blk, int& y) {
    if (!a.nyq_only) {
      blk = t % C::NBLKZ;
      y = t / C::NBLKZ;
    } else if (t < C::NBLKZ) {
      blk = t;
      y = N / 2;
    } else {
      blk = C::NBLKZ - 1;
      y = t - C::NBLKZ;
      if (y >= N / 2) y++;
    }
  };
  const bool mean_in = SC && MODE == Z_FINAL && a.mean == 2;   // previous potential read back
  const bool mean_out = SC && MODE == Z_CURL && a.mean == 1;   // this iteration's potential kept
  auto load = [&](int t, float2* dst, uint64_t* bar) -> uint32_t {
    int blk, y;
    tile_at(t, blk, y);
    if constexpr (MODE == Z_NEWTON) {
      tma::mbar_expect_tx(bar, N * P * 8);
      for (int b = 0; b < C::NBOX; b++)
        tma::load_4d(dst + SOFF + b * C::BOX * P, &in_map, blk * 2 * P, 0, y, b * C::BOX, bar);
      return N * P * 8;
    } else {
      const uint32_t bytes = (mean_in ? 4 : 3) * N * P * 8;
      tma::mbar_expect_tx(bar, bytes);
      for (int b = 0; b < C::NBOX; b++) tma::load_4d(dst + b * C::BOX * VP, &in_map, blk * 2 * P, 0, y, b * C::BOX, bar);
      if (mean_in)
        for (int b = 0; b < C::NBOX; b++)
          tma::load_4d(dst + SOFF + b * C::BOX * P, &phi_map, blk * 2 * P, 3, y, b * C::BOX, bar);
      return bytes;
    }
  };
  auto compute = [&](int t, float2* st) {
    int blk, y;
    tile_at(t, blk, y);
    float2* sv = st;            // vector region
    float2* ss = st + SOFF;     // scalar region
    if constexpr (MODE == Z_NEWTON) fftk::fft<N, -1, P, NTZ>(ss, P, 1, tw, 1, tid);
    else fftk::fft<N, -1, 3 * P, NTZ>(sv, VP, 1, tw, 1, tid);
    const float ky = kv[y], kpy = kp[y];
    const bool ny = (y == N / 2);
    constexpr int PPT = (N * P + NTZ - 1) / NTZ;
    float2 rin[(MODE == Z_NEWTON && !SC) ? PPT : 1];
    if constexpr (MODE == Z_NEWTON && !SC) {
      // the scalar input shares its space with the outputs: read it all first
#pragma unroll
      for (int k = 0; k < PPT; k++) {
        const int i = tid + k * NTZ;
        if (i < N * P) rin[k] = ss[i];
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      const int i = tid + k * NTZ;
      if (i >= N * P) break;
      const int row = i / P, cc = i % P, col = blk * P + cc;
      if (col > N / 2) continue;
      float2* v = sv + row * VP + cc;  // component c at v[c * P]
      float2* sc = ss + row * P + cc;
      const float kx = kv[col], kz = kv[row];
      const bool nx = (col == N / 2), nz = (row == N / 2);
      const float kk = kx * kx + ky * ky + kz * kz;
      const float A = kk > 0.f ? __frcp_rn(kk) : 0.f;  // correctly rounded, as 1.0f / kk
      if constexpr (MODE == Z_NEWTON) {
        float2 r;
        if constexpr (SC) r = *sc;
        else r = rin[k];
        const float f = a.coef * A * a.norm;  // 4 pi G A / N^3
        const float2 ir = cmul_i<1>(r);
        v[0] = cscale(ir, f * kp[col]);
        v[P] = cscale(ir, f * kpy);
        v[2 * P] = cscale(ir, f * kp[row]);
        if constexpr (SC) *sc = cscale(r, -f);  // phi_N^ = -4 pi G A rho^
      } else if constexpr (MODE == Z_SMOOTH) {
        const float f = a.khat[((int64_t)row * N + y) * (N / 2 + 1) + col] * a.norm;
        for (int c = 0; c < 3; c++) v[c * P] = cscale(v[c * P], f);
      } else {
        const float2 gg[3] = {v[0], v[P], v[2 * P]};
        const float k3[3] = {kx, ky, kz};
        const bool n3[3] = {nx, ny, nz};
        if constexpr (MODE == Z_FINAL) {
          // phi^ = i A sum_b k'_b g_b (k'_b = 0 on b's Nyquist plane); a^ = -i kappa phi^
          float2 S = make_float2(0.f, 0.f);
          for (int b = 0; b < 3; b++)
            if (!n3[b]) S = cadd(S, cscale(gg[b], k3[b]));
          float2 aS = cscale(S, A * a.norm);
          if (mean_in) aS = cscale(cadd(aS, *sc), 0.5f);  // the midpoint of the last two iterations
          // times the smoothing spectrum when the mesh is to hold the node-smoothed field
          const float fk = a.khat ? a.khat[((int64_t)row * N + y) * (N / 2 + 1) + col] : 1.0f;
          const float2 aK = cscale(aS, fk);
          v[0] = cscale(aK, kp[col]);
          v[P] = cscale(aK, kpy);
          v[2 * P] = cscale(aK, kp[row]);
          if constexpr (SC) *sc = cmul_i<1>(aS);
        } else if (!(nx || ny || nz)) {
          // away from the Nyquist planes (all but a few per cent of the points):
          // P g = k (k.g) A, from one dot product
          const float2 S = cadd(cadd(cscale(gg[0], kx), cscale(gg[1], ky)), cscale(gg[2], kz));
          const float2 SA = cscale(S, A);
          if (mean_out) *sc = cscale(SA, a.norm);  // the potential this step implies, as Z_FINAL forms it
#pragma unroll
          for (int aa = 0; aa < 3; aa++) {
            const float2 acc = cscale(SA, k3[aa]);
            v[aa * P] = cscale((MODE == Z_DIV) ? csub(gg[aa], acc) : acc, a.norm);
          }
        } else {
          if (mean_out) {
            // the potential this curl-free step implies, as Z_FINAL forms it: A sum_b k'_b g_b
            float2 S = make_float2(0.f, 0.f);
            for (int b = 0; b < 3; b++)
              if (!n3[b]) S = cadd(S, cscale(gg[b], k3[b]));
            *sc = cscale(S, A * a.norm);
          }
          // P_ab = k_a k_b A, off-diagonal terms dropped when exactly one of a, b is on its Nyquist plane
          for (int aa = 0; aa < 3; aa++) {
            float2 acc = make_float2(0.f, 0.f);
            for (int b = 0; b < 3; b++)
              if (aa == b || n3[aa] == n3[b]) acc = cadd(acc, cscale(gg[b], k3[aa] * k3[b] * A));
            v[aa * P] = cscale((MODE == Z_DIV) ? csub(gg[aa], acc) : acc, a.norm);
          }
        }
      }
    }
    __syncthreads();
    fftk::fft<N, +1, 3 * P, NTZ>(sv, VP, 1, tw, 1, tid);
    if (phi) fftk::fft<N, +1, P, NTZ>(ss, P, 1, tw, 1, tid);
  };
  auto store = [&](int t, const float2* src) {
    int blk, y;
    tile_at(t, blk, y);
    const tma::TensorMap* m = SCALAR ? &out_map : &in_map;
    for (int b = 0; b < C::NBOX; b++) tma::store_4d(m, blk * 2 * P, 0, y, b * C::BOX, src + b * C::BOX * VP);
    if (phi || mean_out)
      for (int b = 0; b < C::NBOX; b++)
        tma::store_4d(&phi_map, blk * 2 * P, 3, y, b * C::BOX, src + N * VP + b * C::BOX * P);
  };
  pipe_run(ntiles, stage0, SE, bars, a.status, load, compute, store);
}

// ---------------------------------------------------------------------------
// Folded passes around the curl-free, final and Newton z-passes.
//
// Away from the Nyquist planes the curl-free projection is the gradient of one
// scalar, k (k.g) A, and the final and Newton operators are gradients too
// (-i kappa phi^). So the y-pass before such a z-pass folds the x and y
// components into s = kx gx^ + ky gy^ (component 0; component 2 keeps gz^),
// the z-pass reads two components instead of three and writes the scalar u
// and its z-derivative (components 0 and 2), and the y-pass after it unfolds
// them into the three components again: kx u and ky u before its inverse
// transform, the z one as it is.
//
// Where the Nyquist rule of the projection splits the axes into two sets (a
// point on the kx = N/2 column or the ky = N/2 row) nothing is folded: the
// fold stores gx^ and gy^ apart (the whole y-block holding kx = N/2; for the
// other blocks the row ky = N/2, gy^ written to component 1 of that row
// alone), k_zpass_pipe transforms the z-tiles holding kx = N/2 or ky = N/2
// as it always does (nyq_only), and the unfold takes those values as they
// are. The Newton step has no Nyquist rule (kappa vanishes there), so all its
// tiles are folded. The z-block and the y-block holding kx = N/2 start at the
// same column (fold_ok) so that the passes agree on which columns are apart.
// ---------------------------------------------------------------------------
// kx columns per folded tile of the folded y-passes: two components of
// pyf columns, as many values as a plain tile of pipe_py(n) = 2 pyf columns
constexpr int pipe_pyf(int n) { return pipe_py(n) / 2; }
constexpr int yf_threads(int) { return NT; }

constexpr bool fold_ok(int n) {
  return n >= 32 && ((n / 2) / pipe_pyf(n)) * pipe_pyf(n) == ((n / 2) / pipe_pz(n)) * pipe_pz(n);
}

enum YFoldKind {
  YF_FOLD = 0,   // forward: s = kx gx^ + ky gy^ into component 0
  YF_CURL = 1,   // inverse after the curl-free z-pass: k_x u, k_y u (spectral k)
  YF_GRADN = 2,  // inverse after the final z-pass: kappa_x u, kappa_y u
  YF_GRAD = 3    // inverse after the Newton z-pass: as YF_GRADN, every row and block folded
};

struct PipeYFArgs {
  int nplain;        // components transformed as they are: 2 .. 1 + nplain
  const float2* tw;
  const float* kt;   // per index: k (fold, curl) or kappa (gradients)
  float2* spec;      // the spectral planes (component 1's row ky = N/2: plain loads and stores)
  int64_t pstride;   // complex elements between components
  uint32_t* status;
  int max_ctas;      // cap on the persistent grid (0: as many as fit the GPU)
};

// Tiles of N x PP complex values (PP = pipe_py(N) = 2 pyf, 32 KB at N = 256,
// the plain y-pass's tile): a plain tile holds PP columns of one component;
// a folded tile holds pyf columns of components 0 and 1 interleaved per row,
// [row][component][pyf], loaded and stored through a 4-D view with the
// component as a dimension, so that all tiles take the same conflict-free
// transform. The folded value s (fold) or u (unfold) travels as a compact
// [row][pyf] block of component 0, packed and unpacked in place in two halves.
template <int N, int KIND, int NTY = yf_threads(N)>
__global__ void __launch_bounds__(NTY, 3) k_ypass_fold(const __grid_constant__ tma::TensorMap map4,
                                                    const __grid_constant__ tma::TensorMap mapc,
                                                    const __grid_constant__ tma::TensorMap mapp, PipeYFArgs a) {
  constexpr int PF = pipe_pyf(N), PP = 2 * PF;
  constexpr int H = N / 2;
  constexpr int NBF = (H + 1 + PF - 1) / PF;  // folded blocks; the last holds kx = N/2
  constexpr int NBP = (H + 1 + PP - 1) / PP;  // plain blocks
  constexpr int SP = N / 2 + 2;
  constexpr int BOX = pipe_box(N), NBOX = N / BOX;
  constexpr int DIR = KIND == YF_FOLD ? -1 : +1;
  constexpr int R = N * PP;   // elements of a stage
  constexpr int RC = N * PF;  // elements of a compact block
  constexpr int PER = R / 2 / NTY;  // slots per thread in each half of the tile
  static_assert(R % (2 * NTY) == 0 && NTY % PP == 0 && PP <= 32, "slots split evenly, a warp on whole rows");
  extern __shared__ __align__(128) float2 psm[];
  __shared__ __align__(8) uint64_t bars[2];
  float2* tw = psm;
  float* kt = reinterpret_cast<float*>(psm + N);
  float2* stage0 = psm + 2 * N;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += NTY) {
    tw[i] = a.tw[i];
    kt[i] = a.kt[i];
  }
  const int nxy = NBF * N;
  const int ntiles = nxy + NBP * N * a.nplain;
  // tile -> block, z and component (-1: the folded pair)
  auto decode = [&](int t, int& blk, int& z, int& comp) {
    if (t < nxy) {
      blk = t % NBF;
      z = t / NBF;
      comp = -1;
    } else {
      const int u = t - nxy, rest = u / NBP;
      blk = u % NBP;
      comp = 2 + rest / N;
      z = rest % N;
    }
  };
  // whether a folded tile moves both components whole (else the compact block)
  auto whole = [&](int blk) { return KIND == YF_FOLD ? false : (KIND != YF_GRAD && blk == NBF - 1); };
  auto load = [&](int t, float2* dst, uint64_t* bar) -> uint32_t {
    int blk, z, comp;
    decode(t, blk, z, comp);
    if (comp >= 0) {
      tma::mbar_expect_tx(bar, R * 8);
      for (int b = 0; b < NBOX; b++) tma::load_3d(dst + b * BOX * PP, &mapp, blk * 2 * PP, b * BOX, comp * N + z, bar);
      return R * 8;
    }
    if (KIND == YF_FOLD || whole(blk)) {
      tma::mbar_expect_tx(bar, R * 8);
      for (int b = 0; b < NBOX; b++) tma::load_4d(dst + b * BOX * PP, &map4, blk * 2 * PF, 0, b * BOX, z, bar);
      return R * 8;
    }
    tma::mbar_expect_tx(bar, RC * 8);
    for (int b = 0; b < NBOX; b++) tma::load_3d(dst + b * BOX * PF, &mapc, blk * 2 * PF, b * BOX, z, bar);
    return RC * 8;
  };
  auto compute = [&](int t, float2* st) {
    int blk, z, comp;
    decode(t, blk, z, comp);
    float2* row1 = a.spec + a.pstride + ((int64_t)z * N + H) * SP;  // component 1, row ky = N/2
    // per-element steps over the slots of the tile, a warp on two whole rows
    // (lane q of a row: component q / PF, column q % PF)
    const int q = tid % PP, c = q % PF;
    const bool xs = q < PF;  // the x component's slot
    const float kxc = kt[blk * PF + c];
    if (comp < 0 && KIND != YF_FOLD && !whole(blk)) {
      // unpack u: rows N/2.. first (their slots lie above every packed value),
      // then rows ..N/2 - 1 (read all, then write)
#pragma unroll
      for (int half = 1; half >= 0; half--) {
        float2 u[PER];
#pragma unroll
        for (int k = 0; k < PER; k++) {
          const int row = (half * (R / 2) + tid + k * NTY) / PP;
          u[k] = st[row * PF + c];
        }
        if (half == 0) __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; k++) {
          const int j = half * (R / 2) + tid + k * NTY, row = j / PP;
          if (KIND != YF_GRAD && row == H)  // the Nyquist row: both outputs as the z-pass left them
            st[j] = xs ? u[k] : row1[blk * PF + c];
          else
            st[j] = cscale(u[k], xs ? kxc : kt[row]);
        }
      }
      __syncthreads();
    }
    fftk::fft<N, DIR, PP, NTY>(st, PP, 1, tw, 1, tid);
    if (comp < 0 && KIND == YF_FOLD && blk != NBF - 1) {
      // s = kx gx^ + ky gy^, packed: rows ..N/2 - 1 first (their packed places
      // lie below every unread slot of the second half), then the rest; the
      // y value reaches the x slot's lane by a shuffle
#pragma unroll
      for (int half = 0; half < 2; half++) {
        float2 v[PER];
#pragma unroll
        for (int k = 0; k < PER; k++) {
          const int j = half * (R / 2) + tid + k * NTY, row = j / PP;
          const float2 mine = st[j];
          const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, mine.x, PF),
                                           __shfl_xor_sync(0xffffffffu, mine.y, PF));
          if (row == H) {
            if (!xs) row1[blk * PF + c] = mine;  // gy^ of the Nyquist row, kept apart
            v[k] = mine;
          } else {
            v[k] = cadd(cscale(mine, kxc), cscale(other, kt[row]));
          }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; k++) {
          const int row = (half * (R / 2) + tid + k * NTY) / PP;
          if (xs) st[row * PF + c] = v[k];
        }
      }
    }
  };
  auto store = [&](int t, const float2* src) {
    int blk, z, comp;
    decode(t, blk, z, comp);
    if (comp >= 0) {
      for (int b = 0; b < NBOX; b++) tma::store_3d(&mapp, blk * 2 * PP, b * BOX, comp * N + z, src + b * BOX * PP);
    } else if (KIND == YF_FOLD && blk != NBF - 1) {
      for (int b = 0; b < NBOX; b++) tma::store_3d(&mapc, blk * 2 * PF, b * BOX, z, src + b * BOX * PF);
    } else {
      for (int b = 0; b < NBOX; b++) tma::store_4d(&map4, blk * 2 * PF, 0, b * BOX, z, src + b * BOX * PP);
    }
  };
  pipe_run(ntiles, stage0, R, bars, a.status, load, compute, store);
}

// Folded z-pass (MODE Z_NEWTON, Z_CURL or Z_FINAL) over the tiles away from
// the Nyquist planes of x and y (all tiles for Newton): it reads the folded
// pair (s, gz^) through a map of components 0 and 2 ([z row][2][column] in
// shared memory) and writes (u, z output) the same way; Newton reads rho^
// (component 0) into the upper half of that region and takes it into
// registers before its outputs overwrite it. The arithmetic per point is that of
// k_zpass_pipe, with the x and y factors (k, or kappa for the gradients) left
// to the unfolding y-pass. SCK: 1 = a scalar region for the mean of the last
// two iterations, 2 = also the potential (its inverse z transform).
template <int N, int MODE, int SCK>
__global__ void __launch_bounds__(128, 6) k_zpass_fold(const __grid_constant__ tma::TensorMap in2,
                                                       const __grid_constant__ tma::TensorMap out2,
                                                       const __grid_constant__ tma::TensorMap phi_map, PipeZArgs a) {
  constexpr int NTZ = 128;
  using C = PipeCfg<N>;
  constexpr int P = C::PZ;
  constexpr int H = N / 2;
  constexpr int R = N * P;
  constexpr int IOFF = R;       // Newton: rho^, in the upper half of the pair's region (read out first)
  constexpr int SOFF = 2 * R;   // scalar region
  constexpr int SE = SOFF + (SCK ? R : 0);
  constexpr int NBR = MODE == Z_NEWTON ? C::NBLKZ : C::NBLKZ - 1;  // column blocks visited
  extern __shared__ __align__(128) float2 psm[];
  __shared__ __align__(8) uint64_t bars[2];
  float2* tw = psm;
  float* kv = reinterpret_cast<float*>(psm + N);
  float* kp = kv + N;
  float2* stage0 = psm + 2 * N;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += NTZ) {
    tw[i] = a.tw[i];
    kv[i] = a.kv[i];
    kp[i] = a.kp[i];
  }
  const int ntiles = MODE == Z_NEWTON ? NBR * N : NBR * (N - 1);
  auto tile_at = [&](int t, int& blk, int& y) {
    blk = t % NBR;
    y = t / NBR;
    if (MODE != Z_NEWTON && y >= H) y++;  // the row ky = N/2 is k_zpass_pipe's
  };
  const bool mean_in = SCK && MODE == Z_FINAL && a.mean == 2;
  const bool mean_out = SCK && MODE == Z_CURL && a.mean == 1;
  auto load = [&](int t, float2* dst, uint64_t* bar) -> uint32_t {
    int blk, y;
    tile_at(t, blk, y);
    const uint32_t bytes = ((MODE == Z_NEWTON ? 1 : 2) + (mean_in ? 1 : 0)) * R * 8;
    tma::mbar_expect_tx(bar, bytes);
    for (int b = 0; b < C::NBOX; b++)
      tma::load_4d(dst + (MODE == Z_NEWTON ? IOFF + b * C::BOX * P : b * C::BOX * 2 * P), &in2, blk * 2 * P, 0, y,
                   b * C::BOX, bar);
    if (mean_in)
      for (int b = 0; b < C::NBOX; b++)
        tma::load_4d(dst + SOFF + b * C::BOX * P, &phi_map, blk * 2 * P, 3, y, b * C::BOX, bar);
    return bytes;
  };
  auto compute = [&](int t, float2* st) {
    int blk, y;
    tile_at(t, blk, y);
    float2* ss = st + SOFF;
    const float ky = kv[y];
    constexpr int PPT = (R + NTZ - 1) / NTZ;
    float2 rin[MODE == Z_NEWTON ? PPT : 1];
    if constexpr (MODE == Z_NEWTON) {
      fftk::fft<N, -1, P, NTZ>(st + IOFF, P, 1, tw, 1, tid);
      // the outputs overwrite the input: take it all into registers first
#pragma unroll
      for (int k = 0; k < PPT; k++) {
        const int i = tid + k * NTZ;
        if (i < R) rin[k] = st[IOFF + i];
      }
      __syncthreads();
    } else {
      fftk::fft<N, -1, 2 * P, NTZ, 1>(st, 2 * P, 1, tw, 1, tid);
    }
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      const int i = tid + k * NTZ;
      if (i >= R) break;
      const int row = i / P, cc = i % P, col = blk * P + cc;
      if (col > H) continue;
      const float kx = kv[col], kz = kv[row];
      const float kk = kx * kx + ky * ky + kz * kz;
      const float A = kk > 0.f ? __frcp_rn(kk) : 0.f;  // correctly rounded, as 1.0f / kk
      float2* v = st + row * 2 * P + cc;  // u (in: s) at v[0], z output (in: gz^) at v[P]
      if constexpr (MODE == Z_NEWTON) {
        const float2 r = rin[k];
        const float f = a.coef * A * a.norm;  // 4 pi G A / N^3
        const float2 ir = cmul_i<1>(r);
        v[0] = cscale(ir, f);
        v[P] = cscale(ir, f * kp[row]);
        if constexpr (SCK) ss[i] = cscale(r, -f);  // phi_N^ = -4 pi G A rho^
      } else {
        const bool nz = (row == H);
        const float2 s = v[0], gz = v[P];
        if constexpr (MODE == Z_CURL) {
          if (!nz) {
            const float2 SA = cscale(cadd(s, cscale(gz, kz)), A);
            if (mean_out) ss[i] = cscale(SA, a.norm);
            v[0] = cscale(SA, a.norm);
            v[P] = cscale(cscale(SA, kz), a.norm);
          } else {
            // kz on its Nyquist plane: z is a set of its own
            if (mean_out) ss[i] = cscale(s, A * a.norm);
            v[0] = cscale(cscale(s, A), a.norm);
            v[P] = cscale(cscale(gz, kz * kz * A), a.norm);
          }
        } else {  // Z_FINAL: phi^ = i A sum_b k'_b g_b (k'_z = 0 on its Nyquist plane), a^ = -i kappa phi^
          const float2 S = nz ? s : cadd(s, cscale(gz, kz));
          float2 aS = cscale(S, A * a.norm);
          if (mean_in) aS = cscale(cadd(aS, ss[i]), 0.5f);  // the midpoint of the last two iterations
          const float fk = a.khat ? a.khat[((int64_t)row * N + y) * (N / 2 + 1) + col] : 1.0f;
          const float2 aK = cscale(aS, fk);
          v[0] = aK;
          v[P] = cscale(aK, kp[row]);
          if constexpr (SCK == 2) ss[i] = cmul_i<1>(aS);
        }
      }
    }
    __syncthreads();
    fftk::fft<N, +1, 2 * P, NTZ, 1>(st, 2 * P, 1, tw, 1, tid);
    if constexpr (SCK == 2) fftk::fft<N, +1, P, NTZ>(ss, P, 1, tw, 1, tid);
  };
  auto store = [&](int t, const float2* src) {
    int blk, y;
    tile_at(t, blk, y);
    for (int b = 0; b < C::NBOX; b++) tma::store_4d(&out2, blk * 2 * P, 0, y, b * C::BOX, src + b * C::BOX * 2 * P);
    if (SCK == 2 || mean_out)
      for (int b = 0; b < C::NBOX; b++)
        tma::store_4d(&phi_map, blk * 2 * P, 3, y, b * C::BOX, src + SOFF + b * C::BOX * P);
  };
  pipe_run(ntiles, stage0, SE, bars, a.status, load, compute, store);
}

}  // namespace passes
