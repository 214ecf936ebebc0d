// apparent.cuh -- densities from a mesh field and the masses they imply.
//
// Eq. apparentdensity (Sect. 2.1): rho = -(div g) / (4 pi G). The Newtonian
// field g_N gives the baryonic density rho_B, the MOND acceleration the
// apparent density rho_A, their difference the phantom density. The
// divergence is the periodic central difference (f[i+1] - f[i-1]) / (2 s) that
// the solver's gradients use. Eq. totalmass: the mass inside a volume is the
// flux of g through its boundary over -4 pi G; for a box of cells the face
// value is the mean of the two cells the face separates, which makes the flux
// equal to the box sum of the density.
//
// Fields are 3 planes (x, y, z components) of n^3 floats, x fastest.
#pragma once
#include <cstdint>

namespace dens {

constexpr int NT = 256;
constexpr int MAX_BINS = 4096;

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// Central-difference divergence (times 2 s) of the 4 cells x..x+3 of row
// (y, z); x is a multiple of 4. Differences of neighbouring values first, then
// the sum over the axes in the order x, y, z.
__device__ __forceinline__ float4 div4(const float* __restrict__ g, int n, int64_t n3, int x, int y, int z) {
  const int64_t row = ((int64_t)z * n + y) * n;
  const float* gx = g;
  const float* gy = g + n3;
  const float* gz = g + 2 * n3;
  const float4 c = ld4(gx + row + x);
  const float xm = __ldg(gx + row + (x == 0 ? n - 1 : x - 1));
  const float xp = __ldg(gx + row + (x + 4 == n ? 0 : x + 4));
  const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
  const int zm = z == 0 ? n - 1 : z - 1, zp = z == n - 1 ? 0 : z + 1;
  const float4 a = ld4(gy + ((int64_t)z * n + ym) * n + x);
  const float4 b = ld4(gy + ((int64_t)z * n + yp) * n + x);
  const float4 e = ld4(gz + ((int64_t)zm * n + y) * n + x);
  const float4 f = ld4(gz + ((int64_t)zp * n + y) * n + x);
  float4 d;
  d.x = ((c.y - xm) + (b.x - a.x)) + (f.x - e.x);
  d.y = ((c.z - c.x) + (b.y - a.y)) + (f.y - e.y);
  d.z = ((c.w - c.y) + (b.z - a.z)) + (f.z - e.z);
  d.w = ((xp - c.z) + (b.w - a.w)) + (f.w - e.w);
  return d;
}

// rho for the 4 cells: scale * div4(g) (minus div4(g2) for the phantom density),
// scale = -1 / (2 s 4 pi G).
__device__ __forceinline__ float4 dens4(const float* __restrict__ g, const float* __restrict__ g2, int n,
                                        int64_t n3, int x, int y, int z, float scale) {
  float4 d = div4(g, n, n3, x, y, z);
  if (g2) {
    const float4 d2 = div4(g2, n, n3, x, y, z);
    d.x -= d2.x;
    d.y -= d2.y;
    d.z -= d2.z;
    d.w -= d2.w;
  }
  d.x *= scale;
  d.y *= scale;
  d.z *= scale;
  d.w *= scale;
  return d;
}

// out = density of every cell; one thread per 4 consecutive cells along x.
__global__ void __launch_bounds__(NT) k_density(int n, const float* __restrict__ g, const float* __restrict__ g2,
                                                float scale, float* __restrict__ out) {
  const int64_t n3 = (int64_t)n * n * n;
  const int64_t q = n3 / 4;
  for (int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x; j < q; j += (int64_t)gridDim.x * NT) {
    const int64_t e = 4 * j;
    const int x = (int)(e % n);
    const int64_t r = e / n;
    const int y = (int)(r % n), z = (int)(r / n);
    reinterpret_cast<float4*>(out)[j] = dens4(g, g2, n, n3, x, y, z, scale);
  }
}

// Shell index of the cell centre (x, y, z) about c: floor(r / dr), r the
// minimum-image distance, cell i at (i - n/2) s. Every operation is rounded
// on its own (no contraction), so that a CPU program evaluating the same
// expression in IEEE double picks the same shell.
__device__ __forceinline__ double min_image(int i, int n, double s, double c, double L) {
  double d = __dsub_rn(__dmul_rn((double)(i - n / 2), s), c);
  return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

// Shell sums of the density times s^3 into bins[0..nbins): one thread per 4
// consecutive cells, runs of one shell summed in a register before a shared
// FP64 add, the block's shells added to the global bins at the end.
__global__ void __launch_bounds__(NT) k_shell_mass(int n, const float* __restrict__ g, const float* __restrict__ g2,
                                                   float scale, double s, double cx, double cy, double cz,
                                                   double dr, int nbins, double* __restrict__ bins) {
  __shared__ double sb[MAX_BINS];
  for (int k = threadIdx.x; k < nbins; k += NT) sb[k] = 0.0;
  __syncthreads();
  const int64_t n3 = (int64_t)n * n * n;
  const int64_t q = n3 / 4;
  const double L = (double)n * s;
  const double s3 = s * s * s;
  for (int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x; j < q; j += (int64_t)gridDim.x * NT) {
    const int64_t e = 4 * j;
    const int x = (int)(e % n);
    const int64_t r = e / n;
    const int y = (int)(r % n), z = (int)(r / n);
    const float4 d = dens4(g, g2, n, n3, x, y, z, scale);
    const double dy = min_image(y, n, s, cy, L), dz = min_image(z, n, s, cz, L);
    const double y2 = __dmul_rn(dy, dy);
    const double z2 = __dmul_rn(dz, dz);
    const float v[4] = {d.x, d.y, d.z, d.w};
    int cur = -1;
    double acc = 0.0;
    for (int t = 0; t < 4; t++) {
      const double dx = min_image(x + t, n, s, cx, L);
      const double rr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), y2), z2));
      const double fk = floor(__ddiv_rn(rr, dr));
      const int k = fk < (double)nbins ? (int)fk : -1;
      if (k != cur) {
        if (cur >= 0) atomicAdd(&sb[cur], acc);
        cur = k;
        acc = 0.0;
      }
      acc += (double)v[t] * s3;
    }
    if (cur >= 0) atomicAdd(&sb[cur], acc);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nbins; k += NT)
    if (sb[k] != 0.0) atomicAdd(&bins[k], sb[k]);
}

// Outward flux of g (minus g2) through the faces of the box of cells lo..hi
// (inclusive, periodic), times s^2, added to *out in FP64. One thread per
// face cell; faces in the order (axis, side), cells within a face row-major.
struct Box {
  int lo[3], w[3];
};

__global__ void __launch_bounds__(NT) k_box_flux(int n, const float* __restrict__ g, const float* __restrict__ g2,
                                                 double s, Box bx, double* __restrict__ out) {
  const int64_t n3 = (int64_t)n * n * n;
  int64_t face[3];
  for (int a = 0; a < 3; a++) face[a] = (int64_t)bx.w[(a + 1) % 3] * bx.w[(a + 2) % 3];
  const int64_t total = 2 * (face[0] + face[1] + face[2]);
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x; t < total; t += (int64_t)gridDim.x * NT) {
    int64_t u = t;
    int a = 0;
    while (u >= 2 * face[a]) {
      u -= 2 * face[a];
      a++;
    }
    const int side = u >= face[a] ? 1 : 0;
    if (side) u -= face[a];
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    const int ib = bx.lo[b] + (int)(u / bx.w[c]);
    const int ic = bx.lo[c] + (int)(u % bx.w[c]);
    int p[3], qq[3];
    const int in_a = side ? bx.lo[a] + bx.w[a] - 1 : bx.lo[a];
    const int out_a = side ? in_a + 1 : in_a - 1;
    p[a] = ((in_a % n) + n) % n;
    qq[a] = ((out_a % n) + n) % n;
    p[b] = qq[b] = ((ib % n) + n) % n;
    p[c] = qq[c] = ((ic % n) + n) % n;
    const int64_t ip = ((int64_t)p[2] * n + p[1]) * n + p[0];
    const int64_t iq = ((int64_t)qq[2] * n + qq[1]) * n + qq[0];
    double v = (double)__ldg(g + a * n3 + ip) + (double)__ldg(g + a * n3 + iq);
    if (g2) v -= (double)__ldg(g2 + a * n3 + ip) + (double)__ldg(g2 + a * n3 + iq);
    acc += (side ? 0.5 : -0.5) * v * s * s;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double ws[NT / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int k = 0; k < NT / 32; k++) sum += ws[k];
    atomicAdd(out, sum);
  }
}

}  // namespace dens
