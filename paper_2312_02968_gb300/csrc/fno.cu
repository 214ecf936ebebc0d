// fno.cu -- the learned warm start (include/mond_fno.h): a Fourier neural
// operator on a coarse grid, forward and backward, BF16 weights with FP32
// accumulation, plus the kernels that move fields between the solver mesh and
// the network grid and the sphere-mixture density used to make training pairs.
//
// The spectral convolution keeps only M modes per axis, so its forward and
// inverse transforms are truncated DFTs, evaluated as one small contraction
// per axis (x: real -> M complex; y, z: n -> 2M). The inverse with weight 1
// and no 1/n^3 is the adjoint of the forward, which the backward pass uses.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "../../include/mond_fno.h"
#include "internal.h"

namespace {

constexpr int TB = 256;

struct Shape {
  int n, C, M, L;
  int64_t V;  // n^3
  int K;      // M (2M)(2M)
  __host__ __device__ int64_t layer_size() const { return (int64_t)C * C + C + 2LL * K * C * C; }
  __host__ __device__ int64_t off_P() const { return 0; }
  __host__ __device__ int64_t off_p() const { return 4LL * C; }
  __host__ __device__ int64_t off_layer(int l) const { return 5LL * C + l * layer_size(); }
  __host__ __device__ int64_t off_W(int l) const { return off_layer(l); }
  __host__ __device__ int64_t off_b(int l) const { return off_layer(l) + (int64_t)C * C; }
  __host__ __device__ int64_t off_R(int l) const { return off_layer(l) + (int64_t)C * C + C; }
  __host__ __device__ int64_t off_Q() const { return off_layer(L); }
  __host__ __device__ int64_t off_q() const { return off_Q() + 3LL * C; }
  __host__ __device__ int64_t count() const { return off_q() + 3; }
};

bool make_shape(const mond_fno_shape& s, Shape* o) {
  if (s.n < 8 || s.n > 128 || s.n % 4 || s.width < 1 || s.width > 32 || s.modes < 1 || 2 * s.modes > s.n ||
      s.layers < 1 || s.layers > 8)
    return false;
  o->n = s.n;
  o->C = s.width;
  o->M = s.modes;
  o->L = s.layers;
  o->V = (int64_t)s.n * s.n * s.n;
  o->K = s.modes * 4 * s.modes * s.modes;
  return true;
}

// Workspace layout for one sample.
struct Work {
  float* v;      // (L+1) x C x V activations (v_0 .. v_L)
  float* z;      // L x C x V pre-activations
  float2* shat;  // L x C x K truncated spectra of v_l
  float2* a;     // C x n x n x M  (x-transformed)
  float2* b;     // C x n x 2M x M (y-transformed)
  float2* c;     // C x K          (z-transformed / mixed)
  float2* d;     // C x K
  float* dv;     // C x V
  float* dv2;    // C x V
  float* dz;     // C x V
};

size_t carve(const Shape& s, char* base, Work* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  const size_t CV = (size_t)s.C * s.V;
  Work t{};
  t.v = (float*)take(sizeof(float) * CV * (s.L + 1));
  t.z = (float*)take(sizeof(float) * CV * s.L);
  t.shat = (float2*)take(sizeof(float2) * (size_t)s.C * s.K * s.L);
  t.a = (float2*)take(sizeof(float2) * (size_t)s.C * s.n * s.n * s.M);
  t.b = (float2*)take(sizeof(float2) * (size_t)s.C * s.n * 2 * s.M * s.M);
  t.c = (float2*)take(sizeof(float2) * (size_t)s.C * s.K);
  t.d = (float2*)take(sizeof(float2) * (size_t)s.C * s.K);
  t.dv = (float*)take(sizeof(float) * CV);
  t.dv2 = (float*)take(sizeof(float) * CV);
  t.dz = (float*)take(sizeof(float) * CV);
  if (w) *w = t;
  return off;
}

__device__ __forceinline__ float bf(const uint16_t* p, int64_t i) {
  return __bfloat162float(__ushort_as_bfloat16(p[i]));
}

// e^{sign 2 pi i m / n} with exact argument reduction of m modulo n.
__device__ __forceinline__ float2 cis(int64_t m, int n, float sign) {
  int r = (int)(((m % n) + n) % n);
  float sn, cs;
  sincospif(2.0f * (float)r / (float)n, &sn, &cs);
  return make_float2(cs, sign * sn);
}
__device__ __forceinline__ int sfreq(int i, int M) { return i < M ? i : i - 2 * M; }

// out[o][v] (+)= sum_i W[o][i] in[i][v] (+ b[o]); transpose uses W[i][o].
__global__ void k_pw(const float* in, int Cin, const uint16_t* W, const uint16_t* b, int Cout, float* out, int64_t V,
                     int accumulate, int transpose) {
  __shared__ float sW[32 * 32];
  __shared__ float sb[32];
  for (int i = threadIdx.x; i < Cin * Cout; i += blockDim.x) {
    const int o = i / Cin, j = i % Cin;
    sW[i] = transpose ? bf(W, (int64_t)j * Cout + o) : bf(W, i);
  }
  for (int o = threadIdx.x; o < Cout; o += blockDim.x) sb[o] = b ? bf(b, o) : 0.f;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    float x[32];
    for (int i = 0; i < Cin; i++) x[i] = in[i * V + v];
    for (int o = 0; o < Cout; o++) {
      float acc = sb[o];
      for (int i = 0; i < Cin; i++) acc = fmaf(sW[o * Cin + i], x[i], acc);
      if (accumulate) out[o * V + v] += acc;
      else out[o * V + v] = acc;
    }
  }
}

// dW[o][i] += sum_v dout[o][v] in[i][v]; db[o] += sum_v dout[o][v].
__global__ void k_wgrad(const float* dout, int Cout, const float* in, int Cin, int64_t V, float* dW, float* db) {
  constexpr int CH = 64;
  __shared__ float so[32][CH], si[32][CH];
  const int npair = Cout * Cin + (db ? Cout : 0);
  float acc[5] = {0, 0, 0, 0, 0};
  for (int64_t v0 = (int64_t)blockIdx.x * CH; v0 < V; v0 += (int64_t)gridDim.x * CH) {
    __syncthreads();
    for (int t = threadIdx.x; t < (Cout + Cin) * CH; t += blockDim.x) {
      const int row = t / CH, col = t % CH;
      const int64_t v = v0 + col;
      const float val = v < V ? (row < Cout ? dout[row * V + v] : in[(row - Cout) * V + v]) : 0.f;
      if (row < Cout) so[row][col] = val;
      else si[row - Cout][col] = val;
    }
    __syncthreads();
    for (int k = 0; k < 5; k++) {
      const int p = threadIdx.x + k * blockDim.x;
      if (p >= npair) break;
      float s = 0.f;
      if (p < Cout * Cin) {
        const int o = p / Cin, i = p % Cin;
        for (int c = 0; c < CH; c++) s = fmaf(so[o][c], si[i][c], s);
      } else {
        const int o = p - Cout * Cin;
        for (int c = 0; c < CH; c++) s += so[o][c];
      }
      acc[k] += s;
    }
  }
  for (int k = 0; k < 5; k++) {
    const int p = threadIdx.x + k * blockDim.x;
    if (p >= npair) break;
    if (p < Cout * Cin) atomicAdd(dW + p, acc[k]);
    else atomicAdd(db + (p - Cout * Cin), acc[k]);
  }
}

// Twiddle table e^{-2 pi i m / n}, m in [0, n), in shared memory (n <= 128);
// e^{+...} is its conjugate. Every thread of the block must call it.
__device__ __forceinline__ void load_twiddles(float2* tw, int n) {
  for (int m = threadIdx.x; m < n; m += blockDim.x) tw[m] = cis(m, n, -1.f);
  __syncthreads();
}

// Truncated forward DFT along x of real lines: out[line][kx] = sum_x in[line][x] e^{-2 pi i kx x/n}.
__global__ void k_dft_x(const float* in, float2* out, int64_t nlines, int n, int M) {
  __shared__ float2 tw[128];
  load_twiddles(tw, n);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlines * M) return;
  const int64_t line = t / M;
  const int kx = (int)(t % M);
  const float* p = in + line * n;
  float2 acc = make_float2(0.f, 0.f);
  int m = 0;
  for (int x = 0; x < n; x++) {
    const float2 w = tw[m];
    acc.x = fmaf(p[x], w.x, acc.x);
    acc.y = fmaf(p[x], w.y, acc.y);
    m += kx;
    if (m >= n) m -= n;
  }
  out[t] = acc;
}

// Truncated DFT along an outer axis: in [B][len][inner] -> out [B][2M][inner]
// with out[b][kp][i] = sum_m in[b][m][i] e^{-2 pi i f(kp) m / n}.
__global__ void k_dft_outer(const float2* in, float2* out, int64_t B, int len, int inner, int M, int n) {
  __shared__ float2 tw[128];
  load_twiddles(tw, n);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = B * 2 * M * inner;
  if (t >= tot) return;
  const int i = (int)(t % inner);
  const int kp = (int)((t / inner) % (2 * M));
  const int64_t b = t / ((int64_t)inner * 2 * M);
  const float2* p = in + b * len * inner + i;
  const int f = (sfreq(kp, M) + n) % n;
  float2 acc = make_float2(0.f, 0.f);
  int e = 0;
  for (int m = 0; m < len; m++) {
    const float2 w = tw[e];
    const float2 x = p[(int64_t)m * inner];
    acc.x += x.x * w.x - x.y * w.y;
    acc.y += x.x * w.y + x.y * w.x;
    e += f;
    if (e >= n) e -= n;
  }
  out[t] = acc;
}

// Inverse along an outer axis: in [B][2M][inner] -> out [B][n][inner],
// out[b][m][i] = sum_kp in[b][kp][i] e^{+2 pi i f(kp) m / n}.
__global__ void k_idft_outer(const float2* in, float2* out, int64_t B, int inner, int M, int n) {
  __shared__ float2 tw[128];
  load_twiddles(tw, n);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = B * n * inner;
  if (t >= tot) return;
  const int i = (int)(t % inner);
  const int m = (int)((t / inner) % n);
  const int64_t b = t / ((int64_t)inner * n);
  const float2* p = in + b * 2 * M * inner + i;
  float2 acc = make_float2(0.f, 0.f);
  for (int kp = 0; kp < 2 * M; kp++) {
    const int e = (int)((((int64_t)sfreq(kp, M) * m) % n + n) % n);
    const float2 w = make_float2(tw[e].x, -tw[e].y);
    const float2 x = p[(int64_t)kp * inner];
    acc.x += x.x * w.x - x.y * w.y;
    acc.y += x.x * w.y + x.y * w.x;
  }
  out[t] = acc;
}

// Real lines from the kept x modes: out[line][x] (+)= scale sum_kx a(kx)
// Re(in[line][kx] e^{+2 pi i kx x/n}), a(0) = 1, a(kx > 0) = a_pos.
__global__ void k_idft_x(const float2* in, float* out, int64_t nlines, int n, int M, float a_pos, float scale,
                         int accumulate) {
  __shared__ float2 tw[128];
  load_twiddles(tw, n);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlines * n) return;
  const int64_t line = t / n;
  const int x = (int)(t % n);
  const float2* p = in + line * M;
  float acc = 0.f;
  int e = 0;
  for (int kx = 0; kx < M; kx++) {
    const float2 v = p[kx];
    // Re(v e^{+i th}) = v.x cos th - v.y sin th, with tw = (cos th, -sin th)
    acc += (kx == 0 ? 1.f : a_pos) * (v.x * tw[e].x + v.y * tw[e].y);
    e += x;
    if (e >= n) e -= n;
  }
  acc *= scale;
  if (accumulate) out[t] += acc;
  else out[t] = acc;
}

// t[c][k] = sum_j R[k][j][c] s[j][k] (complex, bf16 weights).
__global__ void k_mix_fwd(const float2* s, const uint16_t* R, float2* t, int C, int K) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)K * C) return;
  const int k = (int)(id / C), c = (int)(id % C);
  float2 acc = make_float2(0.f, 0.f);
  for (int j = 0; j < C; j++) {
    const int64_t r = (((int64_t)k * C + j) * C + c) * 2;
    const float2 w = make_float2(bf(R, r), bf(R, r + 1));
    acc = make_float2(acc.x + w.x * s[(int64_t)j * K + k].x - w.y * s[(int64_t)j * K + k].y,
                      acc.y + w.x * s[(int64_t)j * K + k].y + w.y * s[(int64_t)j * K + k].x);
  }
  t[(int64_t)c * K + k] = acc;
}

// Backward of the mixing with G_t scaled by a(kx)/V first:
// gs[j][k] = sum_c conj(R[k][j][c]) g[c][k]; dR[k][j][c] += conj(s[j][k]) g[c][k].
__global__ void k_mix_bwd(const float2* gt, const float2* s, const uint16_t* R, float2* gs, float* dR, int C, int K,
                          int M, float invV) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)K * C) return;
  const int k = (int)(id / C), j = (int)(id % C);
  const int kx = k % M;
  const float a = (kx == 0 ? 1.f : 2.f) * invV;
  const float2 sj = s[(int64_t)j * K + k];
  float2 acc = make_float2(0.f, 0.f);
  for (int c = 0; c < C; c++) {
    const float2 g = make_float2(gt[(int64_t)c * K + k].x * a, gt[(int64_t)c * K + k].y * a);
    const int64_t r = (((int64_t)k * C + j) * C + c) * 2;
    const float2 w = make_float2(bf(R, r), bf(R, r + 1));
    acc.x += w.x * g.x + w.y * g.y;  // conj(w) g
    acc.y += w.x * g.y - w.y * g.x;
    dR[r] += sj.x * g.x + sj.y * g.y;  // conj(s) g
    dR[r + 1] += sj.x * g.y - sj.y * g.x;
  }
  gs[(int64_t)j * K + k] = acc;
}

__device__ __forceinline__ float gelu_t(float z, float* dgdz) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * (z + k1 * z * z * z);
  const float th = tanhf(u);
  if (dgdz) *dgdz = 0.5f * (1.f + th) + 0.5f * z * (1.f - th * th) * k0 * (1.f + 3.f * k1 * z * z);
  return 0.5f * z * (1.f + th);
}

__global__ void k_gelu(const float* z, float* v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = gelu_t(z[i], nullptr);
}
__global__ void k_gelu_bwd(const float* z, const float* dv, float* dz, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float d;
    gelu_t(z[i], &d);
    dz[i] = dv[i] * d;
  }
}

__global__ void k_sumsq(const float* t, int64_t n, double* out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)t[i] * t[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void k_loss(const float* y, const float* t, float* dy, int64_t n, const double* tnorm, float weight,
                       double* loss) {
  const double inv = 1.0 / fmax(*tnorm, 1e-300);
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += (double)d * d;
    dy[i] = (float)(2.0 * d * inv) * weight;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv * weight);
}

__global__ void k_adam(int64_t n, float* p, float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
  }
}

__global__ void k_cast(const float* p, uint16_t* q, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = __bfloat16_as_ushort(__float2bfloat16_rn(p[i]));
}

// splitmix64 hash -> uniform in [-1, 1)
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
}

__global__ void k_init(Shape s, uint64_t seed, float* p) {
  const int64_t n = s.count();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float scale = 0.f;  // biases start at zero
    if (i < s.off_p()) scale = sqrtf(1.f / 4.f);
    else if (i >= s.off_Q() && i < s.off_q()) scale = sqrtf(1.f / s.C);
    else if (i >= s.off_layer(0) && i < s.off_Q()) {
      const int64_t r = (i - s.off_layer(0)) % s.layer_size();
      if (r < (int64_t)s.C * s.C) scale = sqrtf(1.f / s.C);
      else if (r >= (int64_t)s.C * s.C + s.C) scale = 1.f / ((float)s.C * s.C);
    }
    p[i] = scale * hash_uniform(seed, (uint64_t)i);
  }
}

// Block means of f^3 cells, ncomp planes.
__global__ void k_coarsen(int N, int n, int ncomp, const float* fine, const float* fine2, float* coarse,
                          const float* scale) {
  const int f = N / n;
  const int64_t nc = (int64_t)n * n * n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * ncomp) return;
  const int c = (int)(t / nc);
  const int64_t v = t % nc;
  const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((int64_t)n * n));
  const float* src = fine + (int64_t)c * N * N * N;
  const float* src2 = fine2 ? fine2 + (int64_t)c * N * N * N : nullptr;
  double acc = 0.0;
  for (int dz = 0; dz < f; dz++)
    for (int dy = 0; dy < f; dy++)
      for (int dx = 0; dx < f; dx++) {
        const int64_t i = ((int64_t)(z * f + dz) * N + (y * f + dy)) * N + (x * f + dx);
        acc += src2 ? 0.5 * ((double)src[i] + (double)src2[i]) : (double)src[i];
      }
  const double d = (double)f * f * f * (scale ? (double)*scale : 1.0);
  coarse[t] = (float)(acc / d);
}

__global__ void k_input(int n, float a0, const float* g, const double* sumsq, float* x, float* scale_out) {
  const int64_t V = (int64_t)n * n * n;
  const float s = (float)sqrt(fmax(*sumsq / (3.0 * V), 1e-60));
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = s;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const float gx = g[v], gy = g[V + v], gz = g[2 * V + v];
    x[v] = gx / s;
    x[V + v] = gy / s;
    x[2 * V + v] = gz / s;
    x[3 * V + v] = 0.25f * log10f(sqrtf(gx * gx + gy * gy + gz * gz) / a0 + 1e-12f);
  }
}

// Trilinear, periodic, cell-centred upsampling times the scale.
__global__ void k_output(int N, int n, const float* y, const float* scale, float* H) {
  const int64_t NF = (int64_t)N * N * N, V = (int64_t)n * n * n;
  const int f = N / n;
  const float s = *scale;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 3 * NF; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / NF);
    const int64_t v = t % NF;
    const int X = (int)(v % N), Y = (int)((v / N) % N), Z = (int)(v / ((int64_t)N * N));
    float fx = (X + 0.5f) / f - 0.5f, fy = (Y + 0.5f) / f - 0.5f, fz = (Z + 0.5f) / f - 0.5f;
    const int x0 = (int)floorf(fx), y0 = (int)floorf(fy), z0 = (int)floorf(fz);
    const float wx = fx - x0, wy = fy - y0, wz = fz - z0;
    float acc = 0.f;
    for (int dz = 0; dz < 2; dz++)
      for (int dy = 0; dy < 2; dy++)
        for (int dx = 0; dx < 2; dx++) {
          const int xx = (x0 + dx + n) % n, yy = (y0 + dy + n) % n, zz = (z0 + dz + n) % n;
          const float w = (dx ? wx : 1 - wx) * (dy ? wy : 1 - wy) * (dz ? wz : 1 - wz);
          acc += w * y[c * V + ((int64_t)zz * n + yy) * n + xx];
        }
    H[t] = s * acc;
  }
}

// Sphere mixture on the mesh (Plummer: 3M/(4 pi a^3) (1 + r^2/a^2)^{-5/2};
// Hernquist: M a / (2 pi r (r + a)^3) with r >= 1/2 px), truncated at rmax.
__global__ void k_mixture(int N, float s, int K, const float* centre, const float* mass, const float* radius,
                          const int* kind, float rmax, float* rho) {
  const int64_t NF = (int64_t)N * N * N;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < NF; v += (int64_t)gridDim.x * blockDim.x) {
    const float X = (float)(v % N) - N / 2, Y = (float)((v / N) % N) - N / 2, Z = (float)(v / ((int64_t)N * N)) - N / 2;
    float acc = 0.f;
    for (int j = 0; j < K; j++) {
      const float dx = X - centre[3 * j], dy = Y - centre[3 * j + 1], dz = Z - centre[3 * j + 2];
      float r = sqrtf(dx * dx + dy * dy + dz * dz);
      if (r > rmax) continue;
      const float a = radius[j], m = mass[j];
      if (kind[j] == 0) {
        const float q = 1.f + r * r / (a * a);
        acc += 3.f * m / (4.f * 3.14159265358979f * a * a * a) * powf(q, -2.5f);
      } else {
        r = fmaxf(r, 0.5f);
        acc += m * a / (2.f * 3.14159265358979f * r * (r + a) * (r + a) * (r + a));
      }
    }
    rho[v] = acc / (s * s * s);
  }
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + TB - 1) / TB); }
unsigned grid_stride(int64_t n) {
  int64_t b = (n + TB - 1) / TB;
  return (unsigned)(b < 4096 ? b : 4096);
}

// Spectral convolution forward: shat <- DFT(v); t <- mix; out (+)= IDFT(t).
void spectral_fwd(const Shape& s, const Work& w, const float* v, float2* shat, const uint16_t* R, float* out,
                  cudaStream_t st) {
  const int n = s.n, M = s.M, C = s.C;
  const int64_t lines = (int64_t)C * n * n;
  k_dft_x<<<blocks_for(lines * M), TB, 0, st>>>(v, w.a, lines, n, M);
  // y: [C n][n][M] -> [C n][2M][M]
  k_dft_outer<<<blocks_for((int64_t)C * n * 2 * M * M), TB, 0, st>>>(w.a, w.b, (int64_t)C * n, n, M, M, n);
  // z: [C][n][2M M] -> [C][2M][2M M]
  k_dft_outer<<<blocks_for((int64_t)C * s.K), TB, 0, st>>>(w.b, shat, C, n, 2 * M * M, M, n);
  k_mix_fwd<<<blocks_for((int64_t)s.K * C), TB, 0, st>>>(shat, R, w.c, C, s.K);
  // inverse: z then y then x (weights 1 / 2, 1/n^3)
  k_idft_outer<<<blocks_for((int64_t)C * n * 2 * M * M), TB, 0, st>>>(w.c, w.b, C, 2 * M * M, M, n);
  k_idft_outer<<<blocks_for((int64_t)C * n * n * M), TB, 0, st>>>(w.b, w.a, (int64_t)C * n, M, M, n);
  k_idft_x<<<blocks_for(lines * n), TB, 0, st>>>(w.a, out, lines, n, M, 2.f, 1.f / (float)s.V, 1);
}

}  // namespace

extern "C" {

int mond_fno_param_count(mond_fno_shape sh, int64_t* count) {
  Shape s;
  if (!count || !make_shape(sh, &s)) return -1;
  *count = s.count();
  return 0;
}

int mond_fno_workspace_bytes(mond_fno_shape sh, size_t* bytes) {
  Shape s;
  if (!bytes || !make_shape(sh, &s)) return -1;
  *bytes = carve(s, nullptr, nullptr);
  return 0;
}

int mond_fno_init(mond_fno_shape sh, uint64_t seed, float* params, void* stream) {
  Shape s;
  if (!params || !make_shape(sh, &s)) return -1;
  k_init<<<grid_stride(s.count()), TB, 0, (cudaStream_t)stream>>>(s, seed, params);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_cast(mond_fno_shape sh, const float* params, uint16_t* pb, void* stream) {
  Shape s;
  if (!params || !pb || !make_shape(sh, &s)) return -1;
  k_cast<<<grid_stride(s.count()), TB, 0, (cudaStream_t)stream>>>(params, pb, s.count());
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_forward(mond_fno_shape sh, const uint16_t* P, const float* x, float* y, void* workspace, void* stream) {
  Shape s;
  if (!P || !x || !y || !workspace || !make_shape(sh, &s)) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  Work w;
  carve(s, (char*)workspace, &w);
  const int C = s.C;
  const int64_t V = s.V, CV = (int64_t)C * V;
  const unsigned gv = grid_stride(V);
  k_pw<<<gv, TB, 0, st>>>(x, 4, P + s.off_P(), P + s.off_p(), C, w.v, V, 0, 0);
  for (int l = 0; l < s.L; l++) {
    const float* vl = w.v + l * CV;
    float* zl = w.z + l * CV;
    k_pw<<<gv, TB, 0, st>>>(vl, C, P + s.off_W(l), P + s.off_b(l), C, zl, V, 0, 0);
    spectral_fwd(s, w, vl, w.shat + (int64_t)l * C * s.K, P + s.off_R(l), zl, st);
    float* vn = w.v + (l + 1) * CV;
    if (l + 1 < s.L) k_gelu<<<grid_stride(CV), TB, 0, st>>>(zl, vn, CV);
    else cudaMemcpyAsync(vn, zl, sizeof(float) * CV, cudaMemcpyDeviceToDevice, st);
  }
  k_pw<<<gv, TB, 0, st>>>(w.v + s.L * CV, C, P + s.off_Q(), P + s.off_q(), 3, y, V, 0, 0);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_backward(mond_fno_shape sh, const uint16_t* P, const float* x, const float* dy, float* grad,
                      void* workspace, void* stream) {
  Shape s;
  if (!P || !x || !dy || !grad || !workspace || !make_shape(sh, &s)) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  Work w;
  carve(s, (char*)workspace, &w);
  const int C = s.C, n = s.n, M = s.M;
  const int64_t V = s.V, CV = (int64_t)C * V, lines = (int64_t)C * n * n;
  const unsigned gv = grid_stride(V);
  const unsigned gw = 152;
  // projection
  k_wgrad<<<gw, TB, 0, st>>>(dy, 3, w.v + s.L * CV, C, V, grad + s.off_Q(), grad + s.off_q());
  k_pw<<<gv, TB, 0, st>>>(dy, 3, P + s.off_Q(), nullptr, C, w.dv, V, 0, 1);
  for (int l = s.L - 1; l >= 0; l--) {
    const float* vl = w.v + l * CV;
    const float* zl = w.z + l * CV;
    if (l + 1 < s.L) k_gelu_bwd<<<grid_stride(CV), TB, 0, st>>>(zl, w.dv, w.dz, CV);
    else cudaMemcpyAsync(w.dz, w.dv, sizeof(float) * CV, cudaMemcpyDeviceToDevice, st);
    // pointwise part
    k_wgrad<<<gw, TB, 0, st>>>(w.dz, C, vl, C, V, grad + s.off_W(l), grad + s.off_b(l));
    k_pw<<<gv, TB, 0, st>>>(w.dz, C, P + s.off_W(l), nullptr, C, w.dv2, V, 0, 1);
    // spectral part: G_t = (a/V) DFT(dz), through the mixing adjoint, back with the adjoint transform
    k_dft_x<<<blocks_for(lines * M), TB, 0, st>>>(w.dz, w.a, lines, n, M);
    k_dft_outer<<<blocks_for((int64_t)C * n * 2 * M * M), TB, 0, st>>>(w.a, w.b, (int64_t)C * n, n, M, M, n);
    k_dft_outer<<<blocks_for((int64_t)C * s.K), TB, 0, st>>>(w.b, w.c, C, n, 2 * M * M, M, n);
    k_mix_bwd<<<blocks_for((int64_t)s.K * C), TB, 0, st>>>(w.c, w.shat + (int64_t)l * C * s.K, P + s.off_R(l), w.d,
                                                            grad + s.off_R(l), C, s.K, M, 1.f / (float)V);
    k_idft_outer<<<blocks_for((int64_t)C * n * 2 * M * M), TB, 0, st>>>(w.d, w.b, C, 2 * M * M, M, n);
    k_idft_outer<<<blocks_for((int64_t)C * n * n * M), TB, 0, st>>>(w.b, w.a, (int64_t)C * n, M, M, n);
    k_idft_x<<<blocks_for(lines * n), TB, 0, st>>>(w.a, w.dv2, lines, n, M, 1.f, 1.f, 1);
    cudaMemcpyAsync(w.dv, w.dv2, sizeof(float) * CV, cudaMemcpyDeviceToDevice, st);
  }
  // lift
  k_wgrad<<<gw, TB, 0, st>>>(w.dv, C, x, 4, V, grad + s.off_P(), grad + s.off_p());
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_loss(int64_t count, const float* y, const float* t, float* dy, float weight, double* loss_acc,
                  void* stream) {
  if (!y || !t || !dy || !loss_acc || count <= 0) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  double* tn = loss_acc + 1;  // scratch slot after the accumulator
  cudaMemsetAsync(tn, 0, sizeof(double), st);
  k_sumsq<<<grid_stride(count), TB, 0, st>>>(t, count, tn);
  k_loss<<<grid_stride(count), TB, 0, st>>>(y, t, dy, count, tn, weight, loss_acc);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_adam(int64_t count, float* p, float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                  int step, void* stream) {
  if (!p || !g || !m || !v || count <= 0 || step < 1) return -1;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<grid_stride(count), TB, 0, (cudaStream_t)stream>>>(count, p, g, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_coarsen(int N, int n, int ncomp, const float* fine, const float* fine2, float* coarse,
                     const float* scale, void* stream) {
  if (!fine || !coarse || n <= 0 || N % n || ncomp < 1) return -1;
  const int64_t tot = (int64_t)n * n * n * ncomp;
  k_coarsen<<<blocks_for(tot), TB, 0, (cudaStream_t)stream>>>(N, n, ncomp, fine, fine2, coarse, scale);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_input(int N, int n, float a0, const float* gN, float* x, float* scale_out, void* stream) {
  if (!gN || !x || !scale_out || n <= 0 || N % n) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t V = (int64_t)n * n * n;
  // coarse g_N into the x buffer's first 3 planes, its sum of squares into the scale slot's neighbour
  k_coarsen<<<blocks_for(3 * V), TB, 0, st>>>(N, n, 3, gN, nullptr, x, nullptr);
  double* acc = reinterpret_cast<double*>(scale_out + 2);  // scale_out must have room for 2 + 2 floats
  cudaMemsetAsync(acc, 0, sizeof(double), st);
  k_sumsq<<<grid_stride(3 * V), TB, 0, st>>>(x, 3 * V, acc);
  k_input<<<grid_stride(V), TB, 0, st>>>(n, a0, x, acc, x, scale_out);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_output(int N, int n, const float* y, const float* scale, float* H, void* stream) {
  if (!y || !scale || !H || n <= 0 || N % n) return -1;
  k_output<<<grid_stride(3LL * N * N * N), TB, 0, (cudaStream_t)stream>>>(N, n, y, scale, H);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_mixture_density(int N, double s, int K, const float* centre, const float* mass, const float* radius,
                             const int* kind, float rmax, float* rho, void* stream) {
  if (!centre || !mass || !radius || !kind || !rho || K < 1 || N < 8) return -1;
  k_mixture<<<grid_stride((int64_t)N * N * N), TB, 0, (cudaStream_t)stream>>>(N, (float)s, K, centre, mass, radius,
                                                                             kind, rmax, rho);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
