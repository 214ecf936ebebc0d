// fft.cuh -- shared-memory Stockham FFT building blocks (FP32).
//
// A length-N transform of NSEQ independent sequences held in shared memory,
// element (position p, sequence q) at s[p * PS + q * SS], computed in place by
// a sequence of radix-R Stockham stages (radices 16, 8, 4, 3, 2). Each
// butterfly is a radix-R DFT in registers; the inter-stage twiddles come from
// a shared table tw[m] = (cos(2 pi m / TN), sin(2 pi m / TN)) read with a
// stride TN / N. DIR = -1 is the forward transform e^{-2 pi i jk/N},
// DIR = +1 the inverse (unnormalised).
#pragma once
#include "common.cuh"

namespace fftk {

// cos/sin(2 pi k / 16), k = 0..7 (exact values of the unit circle at pi/8 steps)
__device__ __forceinline__ float c16(int k) {
  const float v[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f,
                      0.0f, -0.38268343236508978f, -0.70710678118654752f, -0.92387953251128674f};
  return v[k];
}
__device__ __forceinline__ float s16(int k) {
  const float v[8] = {0.0f, 0.38268343236508978f, 0.70710678118654752f, 0.92387953251128674f,
                      1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f};
  return v[k];
}

template <int DIR>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int DIR>
__device__ __forceinline__ void dft3(float2* v) {
  // X1,2 = a - (b+c)/2 +- DIR i (sqrt(3)/2)(b - c)
  const float h = 0.86602540378443865f;
  float2 t1 = cadd(v[1], v[2]);
  float2 t2 = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  float2 d = csub(v[1], v[2]);
  float2 t3 = cmul_i<DIR>(make_float2(h * d.x, h * d.y));
  v[0] = cadd(v[0], t1);
  v[1] = cadd(t2, t3);
  v[2] = csub(t2, t3);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
  float2 t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = cmul_i<DIR>(csub(b, d));
  a = cadd(t0, t2);
  c = csub(t0, t2);
  b = cadd(t1, t3);
  d = csub(t1, t3);
}

template <int DIR>
__device__ __forceinline__ void dft8(float2* v) {
  // decimation in time: two DFT4 on even/odd samples, then W8^k combine
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  const float r = 0.70710678118654752f;
  // W8^1 = (r, DIR r), W8^2 = (0, DIR), W8^3 = (-r, DIR r)
  float2 w1 = cmul(o1, make_float2(r, DIR * r));
  float2 w2 = cmul_i<DIR>(o2);
  float2 w3 = cmul(o3, make_float2(-r, DIR * r));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1);
  v[5] = csub(e1, w1);
  v[2] = cadd(e2, w2);
  v[6] = csub(e2, w2);
  v[3] = cadd(e3, w3);
  v[7] = csub(e3, w3);
}

template <int DIR>
__device__ __forceinline__ void dft16(float2* v) {
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft8<DIR>(e);
  dft8<DIR>(o);
#pragma unroll
  for (int k = 0; k < 8; k++) {
    float2 w = cmul(o[k], make_float2(c16(k), DIR * s16(k)));
    v[k] = cadd(e[k], w);
    v[k + 8] = csub(e[k], w);
  }
}

template <int R, int DIR>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 2) dft2<DIR>(v[0], v[1]);
  else if constexpr (R == 3) dft3<DIR>(v);
  else if constexpr (R == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<DIR>(v);
  else if constexpr (R == 16) dft16<DIR>(v);
}

// One radix-R Stockham stage: butterfly j (0 <= j < N/R) of sequence q reads
// positions j + r N/R, multiplies input r by W^{r k N/(Ns R)} with k = j mod Ns,
// transforms, and writes positions (j / Ns) Ns R + k + r Ns.
// Threads are numbered tid < NT; butterfly g -> (q = g % NSEQ, j = g / NSEQ),
// so neighbouring threads touch neighbouring sequences.
// Row swizzle of the intermediate layout of a two-stage transform (mask M):
// the first stage stores position o in row o ^ ((o / B) & M) with B its
// radix, the second reads it back from there (its B = N / its radix, the same
// number). Consecutive butterflies of the first stage, whose rows lie B apart
// and so start on the same bank, then write rows that start on different
// banks: M = 1 spreads 64-byte rows (8 complex values) over both halves of the
// banks (M = 1 and M = 3 on 96-byte rows measured slower). Rows only move
// within aligned groups of M + 1.
template <int B, int M>
__device__ __forceinline__ int swz(int o) {
  if constexpr (B == 0) return o;
  else return o ^ ((o / B) & M);
}

template <int N, int R, int DIR, int NSEQ, int NT, int SWR = 0, int SWW = 0, int M = 1>
__device__ __forceinline__ void stage(float2* s, int PS, int SS, int Ns, const float2* tw, int twstride, int tid) {
  constexpr int NB = N / R;
  constexpr int TOT = NB * NSEQ;
  constexpr int BPT = (TOT + NT - 1) / NT;
  float2 v[BPT][R];
  const int tstep = (N / (Ns * R)) * twstride;
#pragma unroll
  for (int b = 0; b < BPT; b++) {
    int g = tid + b * NT;
    if (TOT % NT == 0 || g < TOT) {
      int q = g % NSEQ, j = g / NSEQ;
      int k = j % Ns;
      const float2* base = s + q * SS;
#pragma unroll
      for (int r = 0; r < R; r++) v[b][r] = base[swz<SWR, M>(j + r * NB) * PS];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; r++) v[b][r] = cmul(v[b][r], twid<DIR>(tw[r * k * tstep]));
      }
      dftR<R, DIR>(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; b++) {
    int g = tid + b * NT;
    if (TOT % NT == 0 || g < TOT) {
      int q = g % NSEQ, j = g / NSEQ;
      int k = j % Ns;
      int o = (j / Ns) * Ns * R + k;
      float2* base = s + q * SS;
#pragma unroll
      for (int r = 0; r < R; r++) base[swz<SWW, M>(o + r * Ns) * PS] = v[b][r];
    }
  }
  __syncthreads();
}

// As stage, for NC groups of NSEQ sequences: sequence l of group c starts at
// s + c CS + l SS, so the groups (the components of a tile) share the
// stage's two barriers.
template <int N, int R, int DIR, int NSEQ, int NC, int NT>
__device__ __forceinline__ void stage_c(float2* s, int PS, int SS, int CS, int Ns, const float2* tw, int twstride,
                                        int tid) {
  constexpr int NB = N / R;
  constexpr int TOT = NB * NSEQ * NC;
  constexpr int BPT = (TOT + NT - 1) / NT;
  float2 v[BPT][R];
  const int tstep = (N / (Ns * R)) * twstride;
#pragma unroll
  for (int b = 0; b < BPT; b++) {
    int g = tid + b * NT;
    if (TOT % NT == 0 || g < TOT) {
      int q = g % (NSEQ * NC), j = g / (NSEQ * NC);
      int k = j % Ns;
      const float2* base = s + (q / NSEQ) * CS + (q % NSEQ) * SS;
#pragma unroll
      for (int r = 0; r < R; r++) v[b][r] = base[(j + r * NB) * PS];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; r++) v[b][r] = cmul(v[b][r], twid<DIR>(tw[r * k * tstep]));
      }
      dftR<R, DIR>(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; b++) {
    int g = tid + b * NT;
    if (TOT % NT == 0 || g < TOT) {
      int q = g % (NSEQ * NC), j = g / (NSEQ * NC);
      int k = j % Ns;
      int o = (j / Ns) * Ns * R + k;
      float2* base = s + (q / NSEQ) * CS + (q % NSEQ) * SS;
#pragma unroll
      for (int r = 0; r < R; r++) base[(o + r * Ns) * PS] = v[b][r];
    }
  }
  __syncthreads();
}

// Radix plans: product of the stage radices equals N.
template <int N>
struct Plan;
#define MOND_PLAN(NN, A, B, C) \
  template <>                  \
  struct Plan<NN> {            \
    static constexpr int r0 = A, r1 = B, r2 = C; \
  };
MOND_PLAN(8, 8, 1, 1)
MOND_PLAN(16, 16, 1, 1)
MOND_PLAN(24, 8, 3, 1)
MOND_PLAN(32, 8, 4, 1)
MOND_PLAN(48, 16, 3, 1)
MOND_PLAN(64, 8, 8, 1)
MOND_PLAN(96, 8, 4, 3)
MOND_PLAN(128, 16, 8, 1)
MOND_PLAN(192, 16, 4, 3)
MOND_PLAN(256, 16, 16, 1)
MOND_PLAN(384, 16, 8, 3)
MOND_PLAN(512, 8, 8, 8)
#undef MOND_PLAN

// Full in-place transform of NSEQ sequences of length N. The twiddle table
// has TN entries for angle 2 pi m / TN with TN = N * twstride.
// SWZ: swizzle mask of the intermediate rows of a two-stage plan (0: none;
// other plans ignore it).
template <int N, int DIR, int NSEQ, int NT, int SWZ = 0>
__device__ __forceinline__ void fft(float2* s, int PS, int SS, const float2* tw, int twstride, int tid) {
  constexpr int R0 = Plan<N>::r0, R1 = Plan<N>::r1, R2 = Plan<N>::r2;
  constexpr int B = (SWZ && R1 > 1 && R2 == 1 && R0 > SWZ) ? R0 : 0;
  stage<N, R0, DIR, NSEQ, NT, 0, B, SWZ>(s, PS, SS, 1, tw, twstride, tid);
  if constexpr (R1 > 1) stage<N, R1, DIR, NSEQ, NT, B, 0, SWZ>(s, PS, SS, R0, tw, twstride, tid);
  if constexpr (R2 > 1) stage<N, R2, DIR, NSEQ, NT>(s, PS, SS, R0 * R1, tw, twstride, tid);
}

// fft over NC groups of NSEQ sequences (group c at s + c CS), one pass of
// barriers for all groups.
template <int N, int DIR, int NSEQ, int NC, int NT>
__device__ __forceinline__ void fft_c(float2* s, int PS, int SS, int CS, const float2* tw, int twstride, int tid) {
  constexpr int R0 = Plan<N>::r0, R1 = Plan<N>::r1, R2 = Plan<N>::r2;
  stage_c<N, R0, DIR, NSEQ, NC, NT>(s, PS, SS, CS, 1, tw, twstride, tid);
  if constexpr (R1 > 1) stage_c<N, R1, DIR, NSEQ, NC, NT>(s, PS, SS, CS, R0, tw, twstride, tid);
  if constexpr (R2 > 1) stage_c<N, R2, DIR, NSEQ, NC, NT>(s, PS, SS, CS, R0 * R1, tw, twstride, tid);
}

}  // namespace fftk
