// Learned warm start for high-precision queries.
//
// The paper computes every query from the zero start (r = e_s).  A model
// maps a cheap sketch of the source to an initial estimate x; the solver then
// pushes the residual of x, r = (alpha e_s + (1-alpha) x P - x) / alpha, to
// lambda exactly as before (the sweeps of the estimate form start from x), so
// the guarantee ||pi_hat - pi||_1 <= lambda never depends on the model.
//
// Model (all per source, batched over B columns):
//   S = alpha e_s + alpha (1-alpha) e_s P + (1-alpha)^2 e_s P^2   (two Power
//       Iterations, Eq. 3 and Eq. 5, plus the alive mass left at step 2)
//   f = S G, G the n x F standard-normal matrix of Box-Muller on Philox
//       (rows keyed by the caller's node id)
//   h = W3 gelu(W2 gelu(W1 f + b1) + b2) + b3        (F -> H -> H -> R)
//   X = max(0, S + U h) / sum(...)                      (U: n x R basis)
// Weights and U are FP32 masters with BF16 copies feeding tensor-core MMAs
// (mma.sync m16n8k16, FP32 accumulation); training minimises the mean l1
// error against exact vectors with Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "fixconv.cuh"
#include "ppr_internal.cuh"

namespace ppr {

typedef unsigned long long u64;
typedef uint16_t bf16r;  // raw BF16 bits
constexpr unsigned kLanes = 0xffffffffu;
constexpr int kR = 64;   // basis rank (columns of U), fixed by the basis kernels

__device__ __forceinline__ bf16r to_bf16(float x) {
  __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<bf16r*>(&b);
}
__device__ __forceinline__ float from_bf16(bf16r x) {
  return __uint_as_float(((uint32_t)x) << 16);
}
__device__ __forceinline__ uint32_t pack2(bf16r lo, bf16r hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * expf(-0.5f * x * x);
}

// Philox-4x32-10 (Salmon et al., SC'11), as in the walk phase
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ------------------------------------------------------------------ sketch
// S[:, c] = alpha e_s + alpha (1-alpha) e_s P + (1-alpha)^2 e_s P^2 (rows = internal ids)
__global__ void sketch_kernel(const int32_t* __restrict__ src_new, int ncols, int B, const int32_t* __restrict__ out_rp,
                              const int32_t* __restrict__ out_ci, const int32_t* __restrict__ deg, float alpha,
                              float* __restrict__ S) {
  const int c = blockIdx.y;
  if (c >= ncols) return;
  const int32_t s = src_new[c];
  const int32_t ds = deg[s], e0 = out_rp[s];
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) atomicAdd(&S[(size_t)s * B + c], alpha);
    const float w1 = alpha * (1.f - alpha) / (float)ds;
    for (int i = threadIdx.x; i < ds; i += blockDim.x) atomicAdd(&S[(size_t)out_ci[e0 + i] * B + c], w1);
  }
  for (int i = blockIdx.x; i < ds; i += gridDim.x) {
    const int32_t u = out_ci[e0 + i];
    const int32_t du = deg[u], f0 = out_rp[u];
    const float w2 = (1.f - alpha) * (1.f - alpha) / ((float)ds * (float)du);
    for (int j = threadIdx.x; j < du; j += blockDim.x) atomicAdd(&S[(size_t)out_ci[f0 + j] * B + c], w2);
  }
}

// ------------------------------------------------------- random projection
// f[c][j] = sum_u S[u][c] G[orig(u)][j]; G rows by Box-Muller on Philox words
// (key (seed), counter (orig id, j/4, 0x47, 0); pairs (w0,w1) and (w2,w3))
template <int B>
__global__ void __launch_bounds__(256) project_kernel(int32_t n, const float* __restrict__ S,
                                                      const int32_t* __restrict__ old_of_new, uint32_t k0,
                                                      uint32_t k1, float* __restrict__ f) {
  constexpr int F = 128;
  constexpr int JB = 256 / B;  // j-blocks
  constexpr int NJ = F / JB;   // j per thread
  __shared__ float Gs[64][F + 1];
  __shared__ float Ss[64][B];
  const int c = threadIdx.x % B, jb = threadIdx.x / B;
  float acc[NJ];
#pragma unroll
  for (int q = 0; q < NJ; ++q) acc[q] = 0.f;
  __shared__ int row_nz[64];
  for (int64_t r0 = (int64_t)blockIdx.x * 64; r0 < n; r0 += (int64_t)gridDim.x * 64) {
    for (int t = threadIdx.x; t < 64 * B; t += blockDim.x) {
      const int row = t / B, cc = t % B;
      Ss[row][cc] = (r0 + row < n) ? S[(size_t)(r0 + row) * B + cc] : 0.f;
    }
    __syncthreads();
    // the sketch is zero outside the sources' 2-hop balls: G rows are made
    // only where some column of S is nonzero
    if (threadIdx.x < 64) {
      int nz = 0;
      for (int cc = 0; cc < B; ++cc) nz |= Ss[threadIdx.x][cc] != 0.f;
      row_nz[threadIdx.x] = nz;
    }
    __syncthreads();
    // 64 rows x 32 Philox calls, 8 calls per thread
    for (int t = threadIdx.x; t < 64 * (F / 4); t += blockDim.x) {
      const int row = t / (F / 4), q = t % (F / 4);
      const int64_t u = r0 + row;
      float z[4] = {0.f, 0.f, 0.f, 0.f};
      if (u < n && row_nz[row]) {
        const uint4 w = philox10(make_uint4((uint32_t)old_of_new[u], (uint32_t)q, 0x47u, 0u), k0, k1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const float u1 = ((float)ws[2 * p] + 1.f) * 2.3283064365386963e-10f;
          const float u2 = (float)ws[2 * p + 1] * 2.3283064365386963e-10f;
          const float rad = sqrtf(-2.f * logf(u1));
          float sn, cs;
          sincospif(2.f * u2, &sn, &cs);
          z[2 * p] = rad * cs;
          z[2 * p + 1] = rad * sn;
        }
      }
#pragma unroll
      for (int p = 0; p < 4; ++p) Gs[row][4 * q + p] = z[p];
    }
    __syncthreads();
    for (int row = 0; row < 64; ++row) {
      const float sv = Ss[row][c];
      if (sv != 0.f)
#pragma unroll
        for (int q = 0; q < NJ; ++q) acc[q] += sv * Gs[row][jb * NJ + q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NJ; ++q)
    if (acc[q] != 0.f) atomicAdd(&f[c * F + jb * NJ + q], acc[q]);
}

// ------------------------------------------------------------ dense GEMMs
// C[M][N] = sum_k A(m,k) B(k,n) (+ bias[n]), BF16 operands, FP32 accumulation.
// A(m,k) = tA ? A[k*lda+m] : A[m*lda+k];  B(k,n) = tB ? B[n*ldb+k] : B[k*ldb+n].
// One warp per 16 x 8 tile of C.  act = 1 also writes gelu(C) as BF16.
struct GemmArgs {
  int M, N, K;
  const bf16r* A;
  int lda, tA;
  const bf16r* B;
  int ldb, tB;
  float* C;       // FP32 result (pre-activation), ldc = N
  bf16r* Cb;      // optional BF16 copy of the activated (act=1) or plain result
  const float* bias;
  int act;
};

__global__ void gemm_bf16_kernel(GemmArgs g) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int tiles_m = (g.M + 15) / 16, tiles_n = g.N / 8;
  if (warp >= tiles_m * tiles_n) return;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  auto A = [&](int m, int k) -> bf16r {
    if (m >= g.M) return 0;
    return g.tA ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k];
  };
  auto Bv = [&](int k, int nn) -> bf16r { return g.tB ? g.B[(size_t)nn * g.ldb + k] : g.B[(size_t)k * g.ldb + nn]; };
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const int r0 = tm * 16 + lane / 4, kq = (lane % 4) * 2, nn = tn * 8 + lane / 4;
  for (int k0 = 0; k0 < g.K; k0 += 16) {
    uint32_t a[4], b[2];
    a[0] = pack2(A(r0, k0 + kq), A(r0, k0 + kq + 1));
    a[1] = pack2(A(r0 + 8, k0 + kq), A(r0 + 8, k0 + kq + 1));
    a[2] = pack2(A(r0, k0 + kq + 8), A(r0, k0 + kq + 9));
    a[3] = pack2(A(r0 + 8, k0 + kq + 8), A(r0 + 8, k0 + kq + 9));
    b[0] = pack2(Bv(k0 + kq, nn), Bv(k0 + kq + 1, nn));
    b[1] = pack2(Bv(k0 + kq + 8, nn), Bv(k0 + kq + 9, nn));
    mma16816(acc, a, b);
  }
  const int col = tn * 8 + kq;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = r0 + (i >= 2 ? 8 : 0), cc = col + (i & 1);
    if (row >= g.M) continue;
    float v = acc[i] + (g.bias ? g.bias[cc] : 0.f);
    g.C[(size_t)row * g.N + cc] = v;
    if (g.Cb) g.Cb[(size_t)row * g.N + cc] = to_bf16(g.act ? gelu_f(v) : v);
  }
}

__global__ void to_bf16_kernel(int64_t count, const float* __restrict__ x, bf16r* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = to_bf16(x[i]);
}

// transpose a (rows x cols) FP32 matrix into a BF16 (cols x rows) one
__global__ void transpose_bf16_kernel(int rows, int cols, const float* __restrict__ x, bf16r* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows * cols) {
    const int r = i / cols, c = i % cols;
    y[(size_t)c * rows + r] = to_bf16(x[i]);
  }
}

// da = dh * gelu'(a) (FP32 and BF16)
__global__ void gelu_back_kernel(int count, const float* __restrict__ dh, const float* __restrict__ a,
                                 float* __restrict__ da, bf16r* __restrict__ dab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    const float v = dh[i] * gelu_grad_f(a[i]);
    da[i] = v;
    dab[i] = to_bf16(v);
  }
}

// column sums of a (rows x cols) matrix (bias gradients)
__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ x, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cols) {
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += x[(size_t)r * cols + c];
    out[c] = s;
  }
}

// ----------------------------------------------------------- basis passes
// One warp per 16 rows: Z = S + U h^T via MMA (K = R = 64), then:
//   pass 1: sig[c] += max(Z, 0)
//   pass 2: X = max(Z,0)/sig (S if sig = 0); loss += |X - pi|; t[c] += sign(X - pi) X / B
//   pass 3: dZ = (sign(X - pi)/B - t[c]) / sig * [Z > 0]; dZ to BF16; dU = dZ h via MMA
//   pass 4: x0 = X in Q1.63, z0 = x0 (1-alpha)/d for the solver's first sweep
struct BasisArgs {
  int32_t n;
  int32_t ncols;        // live columns (others are padding)
  const bf16r* Ub;      // [n][64]
  const bf16r* hb;      // [B][64]
  const bf16r* hTb;     // [64][B]
  const float* S;       // [n][B]
  const float* pi;      // labels, pi[u * ldpi + c]
  int64_t ldpi;
  float* sig;           // [B]
  float* t;             // [B]
  double* loss;
  bf16r* dZb;           // [n][B]
  float* dU;            // [n][64]
  float invB;
  u64* z0;              // pass 4 output [n][kt]
  int kt;
  const uint64_t* omega;
  float* Xout;          // pass 5 output: X as FP32 [n][B]
  int with_sketch;      // Z = S + U h (1) or Z = U h (0: the model predicts a distribution)
  const u64* xin;       // pass 6: current estimate [n][kt] (Q1.63)
  const u64* mass;      // pass 6: [kt] exact sums of xin
  u64* xout;            // passes 4 and 6: the estimate itself (Q1.63), if not NULL
};

template <int B, int PASS>
__global__ void __launch_bounds__(256) basis_kernel(BasisArgs a) {
  constexpr int NB = B / 8;
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int kq = (lane % 4) * 2;
  float part[NB][2];
  float lpart = 0.f;
#pragma unroll
  for (int j = 0; j < NB; ++j) part[j][0] = part[j][1] = 0.f;
  for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < a.n; tile += nwarps) {
    const int r0 = tile * 16 + lane / 4;
    float acc[NB][4];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < kR / 16; ++ks) {
      uint32_t af[4];
      const int k = ks * 16 + kq;
      const bool v0 = r0 < a.n, v1 = r0 + 8 < a.n;
      af[0] = v0 ? *reinterpret_cast<const uint32_t*>(a.Ub + (size_t)r0 * kR + k) : 0u;
      af[1] = v1 ? *reinterpret_cast<const uint32_t*>(a.Ub + (size_t)(r0 + 8) * kR + k) : 0u;
      af[2] = v0 ? *reinterpret_cast<const uint32_t*>(a.Ub + (size_t)r0 * kR + k + 8) : 0u;
      af[3] = v1 ? *reinterpret_cast<const uint32_t*>(a.Ub + (size_t)(r0 + 8) * kR + k + 8) : 0u;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int col = j * 8 + lane / 4;
        uint32_t bfr[2];
        bfr[0] = *reinterpret_cast<const uint32_t*>(a.hb + (size_t)col * kR + k);
        bfr[1] = *reinterpret_cast<const uint32_t*>(a.hb + (size_t)col * kR + k + 8);
        mma16816(acc[j], af, bfr);
      }
    }
    // element-wise stage on the accumulator layout: (row r0 or r0+8, col j*8 + kq + {0,1})
    float dz[NB][4];
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        dz[j][i] = 0.f;
        const int u = r0 + (i >= 2 ? 8 : 0), c = j * 8 + kq + (i & 1);
        if (u >= a.n || c >= a.ncols) continue;
        // the sketch enters Z only in the sketch form; otherwise it is read
        // only as the fallback of a column whose sum is zero
        const bool need_s = a.with_sketch || (PASS != 1 && !(a.sig[c] > 0.f));
        const float s = need_s ? a.S[(size_t)u * B + c] : 0.f;
        const float z = acc[j][i] + (a.with_sketch ? s : 0.f);
        const float y = fmaxf(z, 0.f);
        if constexpr (PASS == 1) {
          part[j][i & 1] += y;
        } else {
          const float sg = a.sig[c];
          const float X = sg > 0.f ? y / sg : s;
          if constexpr (PASS == 4) {
            const u64 xf = f32_to_ufix_trunc(X);
            const u64 om = a.omega[u];
            const u64 hi = __umul64hi(xf, om), lo = xf * om;
            if (c < a.kt) {
              a.z0[(size_t)u * a.kt + c] = hi + (lo >> 63);
              if (a.xout) a.xout[(size_t)u * a.kt + c] = xf;
            }
          } else if constexpr (PASS == 5) {
            a.Xout[(size_t)u * B + c] = X;
          } else if constexpr (PASS == 6) {
            // x += mu X with mu = 1 - sum x (exact, raw units; no correction when
            // the estimate already holds all the mass); z = x (1-alpha)/d
            if (c < a.kt) {
              const long long mu = (long long)(kFixOneRaw - a.mass[c]);
              const u64 add = mu > 0 ? mul_fix_f32((u64)mu, X) : 0ull;
              const u64 xn = a.xin[(size_t)u * a.kt + c] + add;
              const u64 om = a.omega[u];
              const u64 hi = __umul64hi(xn, om), lo = xn * om;
              a.z0[(size_t)u * a.kt + c] = hi + (lo >> 63);
              if (a.xout) a.xout[(size_t)u * a.kt + c] = xn;
            }
          } else {
            const float diff = X - a.pi[(size_t)u * a.ldpi + c];
            const float gsg = diff > 0.f ? a.invB : (diff < 0.f ? -a.invB : 0.f);
            if constexpr (PASS == 2) {
              lpart += fabsf(diff);
              part[j][i & 1] += gsg * X;
            } else {
              const float dY = sg > 0.f ? (gsg - a.t[c]) / sg : 0.f;
              dz[j][i] = z > 0.f ? dY : 0.f;
            }
          }
        }
      }
    if constexpr (PASS == 3) {
      // dZ to BF16 (row-major [n][B]) and dU = dZ h (A from the accumulator layout, B = h^T)
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int c = j * 8 + kq;
        if (r0 < a.n) *reinterpret_cast<uint32_t*>(a.dZb + (size_t)r0 * B + c) = pack2(to_bf16(dz[j][0]), to_bf16(dz[j][1]));
        if (r0 + 8 < a.n)
          *reinterpret_cast<uint32_t*>(a.dZb + (size_t)(r0 + 8) * B + c) = pack2(to_bf16(dz[j][2]), to_bf16(dz[j][3]));
      }
      float du[kR / 8][4];
#pragma unroll
      for (int jr = 0; jr < kR / 8; ++jr) du[jr][0] = du[jr][1] = du[jr][2] = du[jr][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < NB / 2; ++kk) {
        uint32_t af[4];
        af[0] = pack2(to_bf16(dz[2 * kk][0]), to_bf16(dz[2 * kk][1]));
        af[1] = pack2(to_bf16(dz[2 * kk][2]), to_bf16(dz[2 * kk][3]));
        af[2] = pack2(to_bf16(dz[2 * kk + 1][0]), to_bf16(dz[2 * kk + 1][1]));
        af[3] = pack2(to_bf16(dz[2 * kk + 1][2]), to_bf16(dz[2 * kk + 1][3]));
#pragma unroll
        for (int jr = 0; jr < kR / 8; ++jr) {
          const int r = jr * 8 + lane / 4;
          uint32_t bfr[2];
          bfr[0] = *reinterpret_cast<const uint32_t*>(a.hTb + (size_t)r * B + kk * 16 + kq);
          bfr[1] = *reinterpret_cast<const uint32_t*>(a.hTb + (size_t)r * B + kk * 16 + kq + 8);
          mma16816(du[jr], af, bfr);
        }
      }
#pragma unroll
      for (int jr = 0; jr < kR / 8; ++jr) {
        const int r = jr * 8 + kq;
        if (r0 < a.n) *reinterpret_cast<float2*>(a.dU + (size_t)r0 * kR + r) = make_float2(du[jr][0], du[jr][1]);
        if (r0 + 8 < a.n)
          *reinterpret_cast<float2*>(a.dU + (size_t)(r0 + 8) * kR + r) = make_float2(du[jr][2], du[jr][3]);
      }
    }
  }
  if constexpr (PASS == 1 || PASS == 2) {
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float v = part[j][q];
        v += __shfl_xor_sync(kLanes, v, 4);
        v += __shfl_xor_sync(kLanes, v, 8);
        v += __shfl_xor_sync(kLanes, v, 16);
        if (lane < 4 && v != 0.f) atomicAdd((PASS == 1 ? a.sig : a.t) + j * 8 + kq + q, v);
      }
  }
  if constexpr (PASS == 2) {
#pragma unroll
    for (int off = 16; off; off >>= 1) lpart += __shfl_xor_sync(kLanes, lpart, off);
    if (lane == 0) atomicAdd(a.loss, (double)lpart);
  }
}

// dh[b][r] = sum_u dZ[u][b] U[u][r]: split over row chunks, one warp per 16 b-rows
template <int B>
__global__ void __launch_bounds__(B * 2) dh_kernel(int32_t n, const bf16r* __restrict__ dZb,
                                                   const bf16r* __restrict__ Ub, float* __restrict__ dh) {
  constexpr int CH = 256;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // warp -> b rows [16 warp, 16 warp + 16)
  const int kq = (lane % 4) * 2;
  float acc[kR / 8][4];
#pragma unroll
  for (int j = 0; j < kR / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  const int b0 = warp * 16 + lane / 4;
  for (int64_t u0 = (int64_t)blockIdx.x * CH; u0 < n; u0 += (int64_t)gridDim.x * CH) {
    for (int k0 = 0; k0 < CH; k0 += 16) {
      auto dz = [&](int64_t u, int b) -> bf16r { return u < n ? dZb[(size_t)u * B + b] : (bf16r)0; };
      const int64_t u = u0 + k0 + kq;
      uint32_t af[4];
      af[0] = pack2(dz(u, b0), dz(u + 1, b0));
      af[1] = pack2(dz(u, b0 + 8), dz(u + 1, b0 + 8));
      af[2] = pack2(dz(u + 8, b0), dz(u + 9, b0));
      af[3] = pack2(dz(u + 8, b0 + 8), dz(u + 9, b0 + 8));
#pragma unroll
      for (int j = 0; j < kR / 8; ++j) {
        const int r = j * 8 + lane / 4;
        auto uu = [&](int64_t x) -> bf16r { return x < n ? Ub[(size_t)x * kR + r] : (bf16r)0; };
        uint32_t bfr[2];
        bfr[0] = pack2(uu(u), uu(u + 1));
        bfr[1] = pack2(uu(u + 8), uu(u + 9));
        mma16816(acc[j], af, bfr);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kR / 8; ++j) {
    const int r = j * 8 + kq;
    atomicAdd(&dh[b0 * kR + r], acc[j][0]);
    atomicAdd(&dh[b0 * kR + r + 1], acc[j][1]);
    atomicAdd(&dh[(b0 + 8) * kR + r], acc[j][2]);
    atomicAdd(&dh[(b0 + 8) * kR + r + 1], acc[j][3]);
  }
}

// Adam (Kingma & Ba, 2015) on FP32 masters
__global__ void adam_kernel(int64_t count, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// labels: lab[new(o) * ld + col0 + c] = pi[c * n + o] (float)
__global__ void labels_kernel(int64_t n, int ncols, const double* __restrict__ pi, const int32_t* __restrict__ new_of_old,
                              float* __restrict__ lab, int64_t ld, int64_t col0) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = new_of_old[o];
    for (int c = 0; c < ncols; ++c) lab[u * ld + col0 + c] = (float)pi[(size_t)c * n + o];
  }
}

// X (n x B, internal ids) -> out[c * n + o] float64
__global__ void estimate_out_kernel(int64_t n, int ncols, int B, const float* __restrict__ X,
                                    const int32_t* __restrict__ new_of_old, double* __restrict__ out, int64_t col0) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = new_of_old[o];
    for (int c = 0; c < ncols; ++c) out[(size_t)(col0 + c) * n + o] = (double)X[u * B + c];
  }
}

}  // namespace ppr

// ================================================================== model
using namespace ppr;

struct ppr_model {
  ppr_graph* g = nullptr;
  int F = 128, H = 512, R = kR;
  int L = 0;  // correction passes (0: the estimate replaces the zero start)
  uint64_t seed = 0;
  int64_t n_params = 0, off_b1, off_W2, off_b2, off_W3, off_b3, off_U;
  float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  bf16r *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *Ub = nullptr;
  int64_t step = 0;
  // per-batch scratch (batch of kMaxB columns)
  float *S = nullptr, *f = nullptr, *a1 = nullptr, *a2 = nullptr, *h = nullptr, *dh = nullptr, *d1 = nullptr,
        *d2 = nullptr, *red = nullptr;
  bf16r *fb = nullptr, *h1b = nullptr, *h2b = nullptr, *hb = nullptr, *hTb = nullptr, *dhb = nullptr, *d1b = nullptr,
        *d2b = nullptr, *dZb = nullptr;
  double* loss_d = nullptr;
  int32_t* d_src = nullptr;
  float* labels = nullptr;  // host-provided labels staged on the device
  size_t labels_bytes = 0;
};

namespace ppr {
constexpr int kMaxB = 64;

static ppr_status model_alloc(ppr_model* md) {
  const int64_t n = md->g->n, F = md->F, H = md->H, R = md->R;
  md->off_b1 = F * H;
  md->off_W2 = md->off_b1 + H;
  md->off_b2 = md->off_W2 + H * H;
  md->off_W3 = md->off_b2 + H;
  md->off_b3 = md->off_W3 + H * R;
  md->off_U = md->off_b3 + R;
  md->n_params = md->off_U + n * R;
  const size_t pb = sizeof(float) * md->n_params;
  PPR_CUDA_TRY(cudaMalloc(&md->p, pb));
  PPR_CUDA_TRY(cudaMalloc(&md->m, pb));
  PPR_CUDA_TRY(cudaMalloc(&md->v, pb));
  PPR_CUDA_TRY(cudaMalloc(&md->grad, pb));
  PPR_CUDA_TRY(cudaMalloc(&md->W1b, 2 * F * H));
  PPR_CUDA_TRY(cudaMalloc(&md->W2b, 2 * H * H));
  PPR_CUDA_TRY(cudaMalloc(&md->W3b, 2 * H * R));
  PPR_CUDA_TRY(cudaMalloc(&md->Ub, 2 * n * R));
  const int64_t B = kMaxB;
  PPR_CUDA_TRY(cudaMalloc(&md->S, sizeof(float) * n * B));
  PPR_CUDA_TRY(cudaMalloc(&md->f, sizeof(float) * B * F));
  PPR_CUDA_TRY(cudaMalloc(&md->a1, sizeof(float) * B * H));
  PPR_CUDA_TRY(cudaMalloc(&md->a2, sizeof(float) * B * H));
  PPR_CUDA_TRY(cudaMalloc(&md->h, sizeof(float) * B * R));
  PPR_CUDA_TRY(cudaMalloc(&md->dh, sizeof(float) * B * R));
  PPR_CUDA_TRY(cudaMalloc(&md->d1, sizeof(float) * B * H));
  PPR_CUDA_TRY(cudaMalloc(&md->d2, sizeof(float) * B * H));
  PPR_CUDA_TRY(cudaMalloc(&md->red, sizeof(float) * 4 * B));
  PPR_CUDA_TRY(cudaMalloc(&md->fb, 2 * B * F));
  PPR_CUDA_TRY(cudaMalloc(&md->h1b, 2 * B * H));
  PPR_CUDA_TRY(cudaMalloc(&md->h2b, 2 * B * H));
  PPR_CUDA_TRY(cudaMalloc(&md->hb, 2 * B * R));
  PPR_CUDA_TRY(cudaMalloc(&md->hTb, 2 * B * R));
  PPR_CUDA_TRY(cudaMalloc(&md->dhb, 2 * B * R));
  PPR_CUDA_TRY(cudaMalloc(&md->d1b, 2 * B * H));
  PPR_CUDA_TRY(cudaMalloc(&md->d2b, 2 * B * H));
  PPR_CUDA_TRY(cudaMalloc(&md->dZb, 2 * n * B));
  PPR_CUDA_TRY(cudaMalloc(&md->loss_d, sizeof(double)));
  PPR_CUDA_TRY(cudaMalloc(&md->d_src, sizeof(int32_t) * B));
  return PPR_OK;
}

static void model_release(ppr_model* md) {
  for (void* q : {(void*)md->p, (void*)md->m, (void*)md->v, (void*)md->grad, (void*)md->W1b, (void*)md->W2b,
                  (void*)md->W3b, (void*)md->Ub, (void*)md->S, (void*)md->f, (void*)md->a1, (void*)md->a2,
                  (void*)md->h, (void*)md->dh, (void*)md->d1, (void*)md->d2, (void*)md->red, (void*)md->fb,
                  (void*)md->h1b, (void*)md->h2b, (void*)md->hb, (void*)md->hTb, (void*)md->dhb, (void*)md->d1b,
                  (void*)md->d2b, (void*)md->dZb, (void*)md->loss_d, (void*)md->d_src, (void*)md->labels})
    if (q) cudaFree(q);
}

static ppr_status refresh_bf16(ppr_model* md, cudaStream_t st) {
  const int grid = sm_count() * 4;
  to_bf16_kernel<<<grid, 256, 0, st>>>((int64_t)md->F * md->H, md->p, md->W1b);
  to_bf16_kernel<<<grid, 256, 0, st>>>((int64_t)md->H * md->H, md->p + md->off_W2, md->W2b);
  to_bf16_kernel<<<grid, 256, 0, st>>>((int64_t)md->H * md->R, md->p + md->off_W3, md->W3b);
  to_bf16_kernel<<<grid, 256, 0, st>>>(md->g->n * md->R, md->p + md->off_U, md->Ub);
  PPR_CUDA_TRY(cudaGetLastError());
  return PPR_OK;
}

static void gemm(cudaStream_t st, int M, int N, int K, const bf16r* A, int lda, int tA, const bf16r* B, int ldb,
                 int tB, float* C, bf16r* Cb, const float* bias, int act) {
  GemmArgs ga{M, N, K, A, lda, tA, B, ldb, tB, C, Cb, bias, act};
  const int warps = ((M + 15) / 16) * (N / 8);
  gemm_bf16_kernel<<<(warps + 7) / 8, 256, 0, st>>>(ga);
}

// sketch, projection and MLP forward for ncols sources (internal ids) in a batch of B columns
template <int B>
static ppr_status model_forward(ppr_model* md, const int32_t* src_new_host, int ncols, double alpha, cudaStream_t st) {
  ppr_graph* g = md->g;
  const int64_t n = g->n;
  PPR_CUDA_TRY(cudaMemsetAsync(md->S, 0, sizeof(float) * n * B, st));
  PPR_CUDA_TRY(cudaMemsetAsync(md->f, 0, sizeof(float) * B * md->F, st));
  PPR_CUDA_TRY(cudaMemcpyAsync(md->d_src, src_new_host, sizeof(int32_t) * ncols, cudaMemcpyHostToDevice, st));
  sketch_kernel<<<dim3(64, ncols), 256, 0, st>>>(md->d_src, ncols, B, g->d_out_rp, g->d_out_ci, g->d_deg,
                                                 (float)alpha, md->S);
  project_kernel<B><<<sm_count() * 4, 256, 0, st>>>((int32_t)n, md->S, g->d_old_of_new, (uint32_t)md->seed,
                                                    (uint32_t)(md->seed >> 32), md->f);
  to_bf16_kernel<<<8, 256, 0, st>>>((int64_t)B * md->F, md->f, md->fb);
  const int F = md->F, H = md->H, R = md->R;
  gemm(st, B, H, F, md->fb, F, 0, md->W1b, H, 0, md->a1, md->h1b, md->p + md->off_b1, 1);
  gemm(st, B, H, H, md->h1b, H, 0, md->W2b, H, 0, md->a2, md->h2b, md->p + md->off_b2, 1);
  gemm(st, B, R, H, md->h2b, H, 0, md->W3b, R, 0, md->h, md->hb, md->p + md->off_b3, 0);
  transpose_bf16_kernel<<<(B * R + 255) / 256, 256, 0, st>>>(B, R, md->h, md->hTb);
  PPR_CUDA_TRY(cudaGetLastError());
  return PPR_OK;
}

template <int B, int PASS>
static void basis_pass(ppr_model* md, BasisArgs& ba, cudaStream_t st) {
  basis_kernel<B, PASS><<<sm_count() * 4, 256, 0, st>>>(ba);
}

static BasisArgs basis_args(ppr_model* md, int ncols) {
  BasisArgs ba;
  memset(&ba, 0, sizeof(ba));
  ba.n = (int32_t)md->g->n;
  ba.ncols = ncols;
  ba.Ub = md->Ub;
  ba.hb = md->hb;
  ba.hTb = md->hTb;
  ba.S = md->S;
  ba.sig = md->red;
  ba.t = md->red + kMaxB;
  ba.loss = md->loss_d;
  ba.dZb = md->dZb;
  ba.dU = md->grad + md->off_U;
  ba.with_sketch = md->L == 0;
  return ba;
}

// one forward/backward over a batch of ncols <= 64 sources; labels[u * ld + c] (internal ids)
static ppr_status model_step(ppr_model* md, const int32_t* src_new_host, int ncols, const float* labels, int64_t ld,
                             double alpha, float lr, double* loss_out, cudaStream_t st) {
  constexpr int B = kMaxB;
  const int F = md->F, H = md->H, R = md->R;
  PPR_TRY(model_forward<B>(md, src_new_host, ncols, alpha, st));
  PPR_CUDA_TRY(cudaMemsetAsync(md->red, 0, sizeof(float) * 4 * B, st));
  PPR_CUDA_TRY(cudaMemsetAsync(md->loss_d, 0, sizeof(double), st));
  BasisArgs ba = basis_args(md, ncols);
  ba.pi = labels;
  ba.ldpi = ld;
  ba.invB = 1.f / (float)ncols;
  basis_pass<B, 1>(md, ba, st);
  basis_pass<B, 2>(md, ba, st);
  basis_pass<B, 3>(md, ba, st);
  PPR_CUDA_TRY(cudaMemsetAsync(md->dh, 0, sizeof(float) * B * R, st));
  dh_kernel<B><<<sm_count() * 2, B * 2, 0, st>>>((int32_t)md->g->n, md->dZb, md->Ub, md->dh);
  to_bf16_kernel<<<8, 256, 0, st>>>((int64_t)B * R, md->dh, md->dhb);
  float* gW1 = md->grad;
  float* gb1 = md->grad + md->off_b1;
  float* gW2 = md->grad + md->off_W2;
  float* gb2 = md->grad + md->off_b2;
  float* gW3 = md->grad + md->off_W3;
  float* gb3 = md->grad + md->off_b3;
  // layer 3: h = h2 W3 + b3
  gemm(st, H, R, B, md->h2b, H, 1, md->dhb, R, 0, gW3, nullptr, nullptr, 0);
  colsum_kernel<<<1, 64, 0, st>>>(B, R, md->dh, gb3);
  gemm(st, B, H, R, md->dhb, R, 0, md->W3b, R, 1, md->d2, nullptr, nullptr, 0);  // dh2 = dh W3^T
  gelu_back_kernel<<<(B * H + 255) / 256, 256, 0, st>>>(B * H, md->d2, md->a2, md->d2, md->d2b);
  // layer 2
  gemm(st, H, H, B, md->h1b, H, 1, md->d2b, H, 0, gW2, nullptr, nullptr, 0);
  colsum_kernel<<<(H + 255) / 256, 256, 0, st>>>(B, H, md->d2, gb2);
  gemm(st, B, H, H, md->d2b, H, 0, md->W2b, H, 1, md->d1, nullptr, nullptr, 0);  // dh1 = da2 W2^T
  gelu_back_kernel<<<(B * H + 255) / 256, 256, 0, st>>>(B * H, md->d1, md->a1, md->d1, md->d1b);
  // layer 1
  gemm(st, F, H, B, md->fb, F, 1, md->d1b, H, 0, gW1, nullptr, nullptr, 0);
  colsum_kernel<<<(H + 255) / 256, 256, 0, st>>>(B, H, md->d1, gb1);
  PPR_CUDA_TRY(cudaGetLastError());
  if (lr > 0.f) {
    md->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)md->step), c2 = 1.f - std::pow(b2, (float)md->step);
    // a correction model's basis holds a distribution spanning orders of
    // magnitude: it takes smaller steps than the network
    const float lr_u = md->L > 0 ? lr * 0.01f : lr;
    adam_kernel<<<sm_count() * 8, 256, 0, st>>>(md->off_U, md->p, md->m, md->v, md->grad, lr, b1, b2, 1e-8f, c1, c2);
    adam_kernel<<<sm_count() * 8, 256, 0, st>>>(md->n_params - md->off_U, md->p + md->off_U, md->m + md->off_U,
                                                md->v + md->off_U, md->grad + md->off_U, lr_u, b1, b2, 1e-8f, c1, c2);
    PPR_TRY(refresh_bf16(md, st));
  }
  if (loss_out) {
    double l = 0.0;
    PPR_CUDA_TRY(cudaMemcpyAsync(&l, md->loss_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    PPR_CUDA_TRY(cudaStreamSynchronize(st));
    *loss_out = l / ncols;
  }
  return PPR_OK;
}

// X for ncols sources (pass 1 + normalisation); B columns of scratch
template <int B>
static ppr_status model_estimate_internal(ppr_model* md, const int32_t* src_new_host, int ncols, double alpha,
                                          cudaStream_t st) {
  PPR_TRY(model_forward<B>(md, src_new_host, ncols, alpha, st));
  PPR_CUDA_TRY(cudaMemsetAsync(md->red, 0, sizeof(float) * 4 * kMaxB, st));
  BasisArgs ba = basis_args(md, ncols);
  basis_pass<B, 1>(md, ba, st);
  return PPR_OK;
}

// initial estimate for a solver tile: z0[u * kt + c] = x0 (1-alpha) / d_u in Q1.63
ppr_status warm_start_tile(const void* model, ppr_graph* g, const int32_t* src_new, int ncols, int kt, double alpha,
                           unsigned long long* z0, unsigned long long* x0, cudaStream_t st) {
  ppr_model* md = (ppr_model*)model;
  if (md->g != g) { set_error("warm_start model belongs to another graph"); return PPR_ERR_ARG; }
  PPR_TRY(ensure_alpha(g, alpha, st));
  BasisArgs ba = basis_args(md, ncols);
  ba.z0 = z0;
  ba.xout = x0;
  ba.kt = kt;
  ba.omega = g->d_omega;
  const int grid = sm_count() * 4;
  if (kt <= 16) {
    PPR_TRY(model_estimate_internal<16>(md, src_new, ncols, alpha, st));
    basis_kernel<16, 4><<<grid, 256, 0, st>>>(ba);
  } else if (kt <= 32) {
    PPR_TRY(model_estimate_internal<32>(md, src_new, ncols, alpha, st));
    basis_kernel<32, 4><<<grid, 256, 0, st>>>(ba);
  } else {
    PPR_TRY(model_estimate_internal<64>(md, src_new, ncols, alpha, st));
    basis_kernel<64, 4><<<grid, 256, 0, st>>>(ba);
  }
  PPR_CUDA_TRY(cudaGetLastError());
  return PPR_OK;
}

int warm_correction_passes(const void* model) { return ((const ppr_model*)model)->L; }

// x + mu q for a solver tile, written as z = (x + mu q)(1-alpha)/d into z
ppr_status warm_correct_tile(const void* model, ppr_graph* g, const int32_t* src_new, int ncols, int kt,
                             double alpha, const unsigned long long* x, const unsigned long long* mass,
                             unsigned long long* z, unsigned long long* x_out, cudaStream_t st) {
  ppr_model* md = (ppr_model*)model;
  if (md->g != g) { set_error("warm_start model belongs to another graph"); return PPR_ERR_ARG; }
  BasisArgs ba = basis_args(md, ncols);
  ba.z0 = z;
  ba.xout = x_out;
  ba.kt = kt;
  ba.omega = g->d_omega;
  ba.xin = x;
  ba.mass = mass;
  const int grid = sm_count() * 4;
  if (kt <= 16) {
    PPR_TRY(model_estimate_internal<16>(md, src_new, ncols, alpha, st));
    basis_kernel<16, 6><<<grid, 256, 0, st>>>(ba);
  } else if (kt <= 32) {
    PPR_TRY(model_estimate_internal<32>(md, src_new, ncols, alpha, st));
    basis_kernel<32, 6><<<grid, 256, 0, st>>>(ba);
  } else {
    PPR_TRY(model_estimate_internal<64>(md, src_new, ncols, alpha, st));
    basis_kernel<64, 6><<<grid, 256, 0, st>>>(ba);
  }
  PPR_CUDA_TRY(cudaGetLastError());
  return PPR_OK;
}

// start a correction model at the mean training target: U[u][0] = n * mean_c lab[u][c]
// (the scale cancels in the normalisation), W3[:, 0] = 0 and b3[0] = 1 so that
// h_0 = 1 for every source
__global__ void mean_shape_kernel(int64_t n, int64_t ncols, const float* __restrict__ lab, int R,
                                  float* __restrict__ U) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t c = 0; c < ncols; ++c) s += lab[u * ncols + c];
    U[u * R] = (float)(s / (double)ncols * (double)n);
    for (int k = 1; k < R; ++k) U[u * R + k] = 0.f;
  }
}

// correction labels: lab[new(o) * ld + col0 + c] = (pi - x_L)[c][o] / mu_c
__global__ void correction_labels_kernel(int64_t n, int ncols, const double* __restrict__ pi,
                                         const double* __restrict__ xl, const double* __restrict__ mu,
                                         const int32_t* __restrict__ new_of_old, float* __restrict__ lab, int64_t ld,
                                         int64_t col0) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = new_of_old[o];
    for (int c = 0; c < ncols; ++c) {
      const size_t i = (size_t)c * n + o;
      lab[u * ld + col0 + c] = mu[c] > 0.0 ? (float)((pi[i] - xl[i]) / mu[c]) : 0.f;
    }
  }
}

}  // namespace ppr

// ================================================================== C ABI
extern "C" {

void ppr_model_default_opts(ppr_model_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->feat_dim = 128;
  o->hidden = 512;
  o->rank = 64;
  o->correction_passes = 0;
  o->seed = 0x5eedull;
  o->lr = 1e-3f;
  o->epochs = 20;
  o->alpha = 0.2;
  o->lambda = 1e-8;
}

ppr_status ppr_model_create(ppr_graph* g, const ppr_model_opts* opts, ppr_model** out) {
  clear_error();
  if (!g || !out) { set_error("graph and out must be non-NULL"); return PPR_ERR_ARG; }
  *out = nullptr;
  ppr_model_opts o;
  if (opts) o = *opts; else ppr_model_default_opts(&o);
  if (o.feat_dim != 128 || o.rank != kR || o.hidden < 16 || o.hidden % 16) {
    set_error("model needs feat_dim 128, rank 64 and hidden a multiple of 16");
    return PPR_ERR_ARG;
  }
  ppr_model* md = new ppr_model();
  md->g = g;
  md->F = o.feat_dim;
  md->H = o.hidden;
  md->R = o.rank;
  md->L = o.correction_passes;
  md->seed = o.seed;
  if (md->L < 0 || md->L > 200) {
    delete md;
    set_error("correction_passes must lie in [0, 200]");
    return PPR_ERR_ARG;
  }
  ppr_status s = model_alloc(md);
  if (s != PPR_OK) { model_release(md); delete md; return s; }
  // init: W ~ N(0, 1/fan_in), b = 0, U = 0 (the untrained model returns the sketch)
  std::vector<float> host(md->off_U, 0.f);
  std::mt19937_64 rng(o.seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  auto fill = [&](int64_t off, int64_t rows, int64_t cols) {
    const float sc = 1.f / std::sqrt((float)rows);
    for (int64_t i = 0; i < rows * cols; ++i) host[off + i] = nd(rng) * sc;
  };
  fill(0, md->F, md->H);
  fill(md->off_W2, md->H, md->H);
  fill(md->off_W3, md->H, md->R);
  cudaStream_t st = nullptr;
  // a correction model starts from the uniform distribution: U[:, 0] = 1, b3[0] = 1
  if (md->L > 0) host[md->off_b3] = 1.f;
  std::vector<float> u0;
  if (md->L > 0) {
    u0.assign((size_t)g->n * md->R, 0.f);
    for (int64_t u = 0; u < g->n; ++u) u0[(size_t)u * md->R] = 1.f;
  }
  if (cudaMemcpy(md->p, host.data(), sizeof(float) * host.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(md->p + md->off_U, 0, sizeof(float) * g->n * md->R) != cudaSuccess ||
      (md->L > 0 && cudaMemcpy(md->p + md->off_U, u0.data(), sizeof(float) * u0.size(), cudaMemcpyHostToDevice) !=
                        cudaSuccess) ||
      cudaMemset(md->m, 0, sizeof(float) * md->n_params) != cudaSuccess ||
      cudaMemset(md->v, 0, sizeof(float) * md->n_params) != cudaSuccess ||
      cudaMemset(md->grad, 0, sizeof(float) * md->n_params) != cudaSuccess || refresh_bf16(md, st) != PPR_OK ||
      cudaDeviceSynchronize() != cudaSuccess) {
    set_error("model initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
    model_release(md);
    delete md;
    return PPR_ERR_CUDA;
  }
  *out = md;
  return PPR_OK;
}

void ppr_model_free(ppr_model* md) {
  if (!md) return;
  cudaDeviceSynchronize();
  model_release(md);
  delete md;
}

int64_t ppr_model_param_count(const ppr_model* md) { return md ? md->n_params : 0; }

// parameters (and gradients) in the flat order W1, b1, W2, b2, W3, b3, U with
// U's rows in the caller's node order
ppr_status ppr_model_get_params(const ppr_model* md, float* params, float* grads) {
  clear_error();
  if (!md) { set_error("model is NULL"); return PPR_ERR_ARG; }
  const int64_t n = md->g->n, R = md->R, off = md->off_U;
  std::vector<float> buf(md->n_params);
  for (int which = 0; which < 2; ++which) {
    float* dst = which == 0 ? params : grads;
    if (!dst) continue;
    const float* src = which == 0 ? md->p : md->grad;
    PPR_CUDA_TRY(cudaMemcpy(buf.data(), src, sizeof(float) * md->n_params, cudaMemcpyDeviceToHost));
    memcpy(dst, buf.data(), sizeof(float) * off);
    for (int64_t o = 0; o < n; ++o)
      memcpy(dst + off + o * R, buf.data() + off + (int64_t)md->g->h_new_of_old[o] * R, sizeof(float) * R);
  }
  return PPR_OK;
}

ppr_status ppr_model_set_params(ppr_model* md, const float* params) {
  clear_error();
  if (!md || !params) { set_error("model and params must be non-NULL"); return PPR_ERR_ARG; }
  const int64_t n = md->g->n, R = md->R, off = md->off_U;
  std::vector<float> buf(md->n_params);
  memcpy(buf.data(), params, sizeof(float) * off);
  for (int64_t o = 0; o < n; ++o)
    memcpy(buf.data() + off + (int64_t)md->g->h_new_of_old[o] * R, params + off + o * R, sizeof(float) * R);
  PPR_CUDA_TRY(cudaMemcpy(md->p, buf.data(), sizeof(float) * md->n_params, cudaMemcpyHostToDevice));
  PPR_TRY(refresh_bf16(md, nullptr));
  PPR_CUDA_TRY(cudaDeviceSynchronize());
  return PPR_OK;
}

ppr_status ppr_model_train_step(ppr_model* md, const int32_t* src, int32_t k, const double* labels, float lr,
                                double* loss, void* stream) {
  clear_error();
  if (!md || !src || !labels || k < 1 || k > kMaxB || lr < 0.f) {
    set_error("train_step needs a model, 1..64 sources and labels");
    return PPR_ERR_ARG;
  }
  ppr_graph* g = md->g;
  const int64_t n = g->n;
  for (int i = 0; i < k; ++i)
    if (src[i] < 0 || src[i] >= n) { set_error("source out of range"); return PPR_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  // labels (k x n, caller's order, host or device) -> internal [n][k] FP32
  const size_t lb = sizeof(float) * n * kMaxB;
  if (md->labels_bytes < lb) {
    if (md->labels) cudaFree(md->labels);
    md->labels = nullptr;
    PPR_CUDA_TRY(cudaMalloc(&md->labels, lb));
    md->labels_bytes = lb;
  }
  const double* lab_dev = labels;
  double* staged = nullptr;
  if (!is_device_pointer(labels)) {
    PPR_CUDA_TRY(cudaMalloc(&staged, sizeof(double) * n * k));
    PPR_CUDA_TRY(cudaMemcpyAsync(staged, labels, sizeof(double) * n * k, cudaMemcpyHostToDevice, st));
    lab_dev = staged;
  }
  labels_kernel<<<sm_count() * 4, 256, 0, st>>>(n, k, lab_dev, g->d_new_of_old, md->labels, kMaxB, 0);
  std::vector<int32_t> s_new(k);
  for (int i = 0; i < k; ++i) s_new[i] = g->h_new_of_old[src[i]];
  ppr_status s = model_step(md, s_new.data(), k, md->labels, kMaxB, 0.2, lr, loss, st);
  if (staged) {
    cudaStreamSynchronize(st);
    cudaFree(staged);
  }
  return s;
}

ppr_status ppr_model_estimate(ppr_model* md, const int32_t* src, int32_t k, double* out_x, void* stream) {
  clear_error();
  if (!md || !src || !out_x || k < 1) { set_error("estimate needs a model, sources and an output"); return PPR_ERR_ARG; }
  ppr_graph* g = md->g;
  const int64_t n = g->n;
  for (int i = 0; i < k; ++i)
    if (src[i] < 0 || src[i] >= n) { set_error("source out of range"); return PPR_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const bool host = !is_device_pointer(out_x);
  double* dev = out_x;
  if (host) PPR_CUDA_TRY(cudaMalloc(&dev, sizeof(double) * n * k));
  for (int32_t t0 = 0; t0 < k; t0 += kMaxB) {
    const int nc = std::min<int32_t>(kMaxB, k - t0);
    std::vector<int32_t> s_new(nc);
    for (int i = 0; i < nc; ++i) s_new[i] = g->h_new_of_old[src[t0 + i]];
    PPR_TRY(model_estimate_internal<kMaxB>(md, s_new.data(), nc, 0.2, st));
    const size_t lb = sizeof(float) * n * kMaxB;
    if (md->labels_bytes < lb) {
      if (md->labels) cudaFree(md->labels);
      md->labels = nullptr;
      PPR_CUDA_TRY(cudaMalloc(&md->labels, lb));
      md->labels_bytes = lb;
    }
    BasisArgs ba = basis_args(md, nc);
    ba.Xout = md->labels;
    basis_kernel<kMaxB, 5><<<sm_count() * 4, 256, 0, st>>>(ba);
    estimate_out_kernel<<<sm_count() * 4, 256, 0, st>>>(n, nc, kMaxB, md->labels, g->d_new_of_old, dev, t0);
    PPR_CUDA_TRY(cudaGetLastError());
  }
  if (host) {
    PPR_CUDA_TRY(cudaMemcpyAsync(out_x, dev, sizeof(double) * n * k, cudaMemcpyDeviceToHost, st));
    PPR_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(dev);
  }
  PPR_CUDA_TRY(cudaStreamSynchronize(st));
  return PPR_OK;
}

ppr_status ppr_model_train(ppr_model* md, const int32_t* train_src, int32_t n_src, int32_t epochs, float lr,
                           uint64_t shuffle_seed, float* loss_per_epoch, void* stream) {
  clear_error();
  if (!md || !train_src || n_src < 1 || epochs < 0 || !(lr >= 0.f)) {
    set_error("train needs a model, training sources, epochs >= 0 and lr >= 0");
    return PPR_ERR_ARG;
  }
  ppr_graph* g = md->g;
  const int64_t n = g->n;
  for (int32_t i = 0; i < n_src; ++i)
    if (train_src[i] < 0 || train_src[i] >= n) { set_error("training source out of range"); return PPR_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  // Exact labels from the plain high-precision method, [n][chunk] FP32.  When
  // labels for every source do not fit in half of the free device memory, the
  // sources are taken in chunks whose labels are regenerated every epoch.
  size_t free_b = 0, total_b = 0;
  PPR_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  // label queries use the widest tile whose workspace takes at most 30 % of free memory
  int kt_label = kMaxB;
  while (kt_label > 1 && (double)hp_state_bytes(g, kMaxB, kt_label) > 0.3 * (double)free_b) kt_label /= 2;
  const size_t fixed = 2 * sizeof(double) * n * kMaxB + (size_t)hp_state_bytes(g, kMaxB, kt_label) +
                       ((size_t)1 << 30);
  if (free_b < fixed + sizeof(float) * (size_t)n * kMaxB) {
    set_error("admission refused: training needs at least %zu bytes, %zu free", fixed, free_b);
    return PPR_ERR_ADMIT;
  }
  int32_t chunk = n_src;
  if (sizeof(float) * (size_t)n * n_src > (free_b - fixed) / 2)
    chunk = std::max<int32_t>(kMaxB, (int32_t)(((free_b - fixed) / 2 / (sizeof(float) * (size_t)n)) / kMaxB * kMaxB));
  chunk = std::min(chunk, n_src);
  float* lab = nullptr;
  double* buf = nullptr;
  double* xl = nullptr;
  double* mu_d = nullptr;
  PPR_CUDA_TRY(cudaMalloc(&lab, sizeof(float) * (size_t)n * chunk));
  if (cudaMalloc(&buf, sizeof(double) * n * kMaxB) != cudaSuccess ||
      (md->L > 0 && (cudaMalloc(&xl, sizeof(double) * n * kMaxB) != cudaSuccess ||
                     cudaMalloc(&mu_d, sizeof(double) * kMaxB) != cudaSuccess))) {
    cudaFree(lab); cudaFree(buf); cudaFree(xl);
    set_error("out of device memory for label generation");
    return PPR_ERR_OOM;
  }
  ppr_status s = PPR_OK;
  ppr_query_opts qo;
  ppr_default_opts(&qo);
  qo.alpha = 0.2;
  qo.k_tile = kt_label;
  std::vector<ppr_stats> pst(kMaxB);
  // labels for sources [c0, c0 + cnt) into columns [0, cnt) of lab (ld = chunk)
  auto make_labels = [&](int32_t c0, int32_t cnt) -> ppr_status {
    for (int32_t b = 0; b < cnt; b += kMaxB) {
      const int nc = std::min<int32_t>(kMaxB, cnt - b);
      PPR_TRY(query_hp(g, train_src + c0 + b, nc, qo, buf, nullptr, nullptr, st));
      if (md->L == 0) {
        labels_kernel<<<sm_count() * 4, 256, 0, st>>>(n, nc, buf, g->d_new_of_old, lab, chunk, b);
      } else {
        // target: the distribution of the mass the zero-start solve still misses after L passes
        ppr_query_opts qp = qo;
        qp.max_sweeps = md->L;
        qp.flags = PPR_FLAG_PARTIAL;
        PPR_TRY(query_hp(g, train_src + c0 + b, nc, qp, xl, nullptr, pst.data(), st));
        double mu_h[kMaxB];
        for (int c = 0; c < nc; ++c) mu_h[c] = pst[c].mass_deficit;
        PPR_CUDA_TRY(cudaMemcpyAsync(mu_d, mu_h, sizeof(double) * nc, cudaMemcpyHostToDevice, st));
        correction_labels_kernel<<<sm_count() * 4, 256, 0, st>>>(n, nc, buf, xl, mu_d, g->d_new_of_old, lab, chunk,
                                                                 b);
        PPR_CUDA_TRY(cudaStreamSynchronize(st));
      }
    }
    return PPR_OK;
  };
  auto shape_init = [&](int32_t cnt) -> ppr_status {
    mean_shape_kernel<<<sm_count() * 4, 256, 0, st>>>(n, cnt, lab, md->R, md->p + md->off_U);
    std::vector<float> zero(md->H, 0.f);
    for (int h = 0; h < md->H; ++h)
      PPR_CUDA_TRY(cudaMemcpyAsync(md->p + md->off_W3 + (int64_t)h * md->R, &zero[h], sizeof(float),
                                   cudaMemcpyHostToDevice, st));
    const float one = 1.f;
    PPR_CUDA_TRY(cudaMemcpyAsync(md->p + md->off_b3, &one, sizeof(float), cudaMemcpyHostToDevice, st));
    PPR_CUDA_TRY(cudaStreamSynchronize(st));
    return refresh_bf16(md, st);
  };
  const int nchunks = (n_src + chunk - 1) / chunk;
  std::vector<int> chunk_order(nchunks);
  std::iota(chunk_order.begin(), chunk_order.end(), 0);
  bool labels_ready = false;
  for (int ep = 0; (ep < epochs || (ep == 0 && md->L > 0 && md->step == 0)) && s == PPR_OK; ++ep) {
    std::mt19937_64 rng(shuffle_seed + (uint64_t)ep);
    std::shuffle(chunk_order.begin(), chunk_order.end(), rng);
    double tot = 0.0;
    for (int ci = 0; ci < nchunks && s == PPR_OK; ++ci) {
      const int32_t c0 = chunk_order[ci] * chunk;
      const int32_t cnt = std::min<int32_t>(chunk, n_src - c0);
      if (!labels_ready) s = make_labels(c0, cnt);
      if (s != PPR_OK) break;
      if (nchunks == 1) labels_ready = true;
      // a correction model starts at the mean target of the first labels it sees
      if (md->L > 0 && md->step == 0) s = shape_init(cnt);
      if (s != PPR_OK || ep >= epochs) break;
      const int nb = (cnt + kMaxB - 1) / kMaxB;
      std::vector<int> order(nb);
      std::iota(order.begin(), order.end(), 0);
      std::shuffle(order.begin(), order.end(), rng);
      for (int bi = 0; bi < nb && s == PPR_OK; ++bi) {
        const int b0 = order[bi] * kMaxB;
        const int nc = std::min<int32_t>(kMaxB, cnt - b0);
        std::vector<int32_t> s_new(nc);
        for (int i = 0; i < nc; ++i) s_new[i] = g->h_new_of_old[train_src[c0 + b0 + i]];
        double l = 0.0;
        s = model_step(md, s_new.data(), nc, lab + b0, chunk, 0.2, lr, &l, st);
        tot += l * nc;
      }
    }
    if (loss_per_epoch && ep < epochs) loss_per_epoch[ep] = (float)(tot / n_src);
  }
  cudaFree(buf);
  if (xl) cudaFree(xl);
  if (mu_d) cudaFree(mu_d);
  cudaStreamSynchronize(st);
  cudaFree(lab);
  return s;
}

// checkpoint: magic, version, n, F, H, R, seed, step, correction passes, then
// parameters and both Adam moments
ppr_status ppr_model_save(const ppr_model* md, const char* path) {
  clear_error();
  if (!md || !path) { set_error("model and path must be non-NULL"); return PPR_ERR_ARG; }
  FILE* fp = fopen(path, "wb");
  if (!fp) { set_error("cannot open %s for writing", path); return PPR_ERR_ARG; }
  const int64_t hdr[9] = {0x4d525050, 2, md->g->n, md->F, md->H, md->R, (int64_t)md->seed, md->step, md->L};
  std::vector<float> buf(md->n_params);
  bool io_ok = fwrite(hdr, sizeof(hdr), 1, fp) == 1, cuda_ok = true;
  for (const float* src : {md->p, md->m, md->v}) {
    if (!io_ok) break;
    cuda_ok = cudaMemcpy(buf.data(), src, sizeof(float) * md->n_params, cudaMemcpyDeviceToHost) == cudaSuccess;
    io_ok = cuda_ok && fwrite(buf.data(), sizeof(float), md->n_params, fp) == (size_t)md->n_params;
  }
  io_ok = (fclose(fp) == 0) && io_ok;
  if (!cuda_ok) { set_error("copying the model from the device failed"); return PPR_ERR_CUDA; }
  if (!io_ok) { set_error("writing %s failed", path); return PPR_ERR_ARG; }
  return PPR_OK;
}

ppr_status ppr_model_load(ppr_graph* g, const char* path, ppr_model** out) {
  clear_error();
  if (!g || !path || !out) { set_error("graph, path and out must be non-NULL"); return PPR_ERR_ARG; }
  *out = nullptr;
  FILE* fp = fopen(path, "rb");
  if (!fp) { set_error("cannot open %s", path); return PPR_ERR_ARG; }
  int64_t hdr[9];
  if (fread(hdr, sizeof(hdr), 1, fp) != 1 || hdr[0] != 0x4d525050 || hdr[1] != 2 || hdr[2] != g->n) {
    fclose(fp);
    set_error("%s is not a model checkpoint for this graph", path);
    return PPR_ERR_ARG;
  }
  ppr_model_opts o;
  ppr_model_default_opts(&o);
  o.feat_dim = (int32_t)hdr[3];
  o.hidden = (int32_t)hdr[4];
  o.rank = (int32_t)hdr[5];
  o.seed = (uint64_t)hdr[6];
  o.correction_passes = (int32_t)hdr[8];
  ppr_model* md = nullptr;
  ppr_status s = ppr_model_create(g, &o, &md);
  if (s != PPR_OK) { fclose(fp); return s; }
  std::vector<float> buf(md->n_params);
  bool ok = true;
  for (float* dst : {md->p, md->m, md->v}) {
    if (!ok) break;
    ok = fread(buf.data(), sizeof(float), md->n_params, fp) == (size_t)md->n_params &&
         cudaMemcpy(dst, buf.data(), sizeof(float) * md->n_params, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  fclose(fp);
  md->step = hdr[7];
  if (!ok || refresh_bf16(md, nullptr) != PPR_OK || cudaDeviceSynchronize() != cudaSuccess) {
    ppr_model_free(md);
    set_error("reading %s failed", path);
    return PPR_ERR_ARG;
  }
  *out = md;
  return PPR_OK;
}

}  // extern "C"
