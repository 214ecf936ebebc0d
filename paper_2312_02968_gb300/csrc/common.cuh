// common.cuh -- shared definitions of the CUDA path (device helpers, status
// bits, workspace layout structs). Nothing here is shared with the CPU oracle.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define MOND_HD __host__ __device__ __forceinline__

// Device status bits, OR-ed into a word in the workspace and read at
// synchronising calls.
enum : uint32_t {
  ST_DOMAIN = 1u,    // particle cell/offset outside the domain (skipped)
  ST_NAN = 2u,       // non-finite value in a field or particle
  ST_TIMEOUT = 4u,   // a bounded device wait gave up
  ST_OVERFLOW = 8u,  // fixed-point bound violated
};

// ---------------------------------------------------------------------------
// Complex arithmetic on float2 (x = real, y = imaginary).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (DIR * i): DIR = -1 gives a * (-i), DIR = +1 gives a * i
template <int DIR>
__device__ __forceinline__ float2 cmul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
// e^{DIR * i * theta} from the table entry (cos theta, sin theta)
template <int DIR>
__device__ __forceinline__ float2 twid(float2 t) {
  return DIR < 0 ? make_float2(t.x, -t.y) : t;
}

// signed frequency of index i on an axis of length n (Nyquist n/2 -> -n/2)
MOND_HD int freq_of(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

__device__ __forceinline__ int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ void set_status(uint32_t* st, uint32_t bit) { atomicOr(st, bit); }

// ---------------------------------------------------------------------------
// Mesh geometry passed by value to every pass.
// ---------------------------------------------------------------------------
struct MeshGeom {
  int n;          // FFT-domain side n_f
  int sp;         // spectral row stride in complex elements (n/2 + 2)
  int64_t plane;  // spectral plane stride in complex elements (n * n * sp)
  int64_t cells;  // n^3
  float s;        // pixel width
};
