// lcnn_kernels.cu -- kernels of the learned warm start: a small 3D U-Net that
// proposes the relaxed Q around a colloid, trained on fields the solver
// itself relaxes.  Activations are channels-last BF16 ([position][channel],
// position = x + W*(y + H*z)), weights [C_out][taps][C_in] BF16 with FP32
// masters; every convolution accumulates in FP32 on the tensor cores
// (mma.sync m16n8k16 bf16, implicit GEMM).  Boundaries are periodic, like the
// boxes the fields come from.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lc_nn.h"

namespace lcnn {

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Position of tap t (0..26, (dz+1)*9 + (dy+1)*3 + (dx+1)) around p; taps == 1: p itself.
__device__ __forceinline__ int tap_pos(int p, int t, int taps, int W, int H, int D) {
  if (taps == 1) return p;
  const int x = p % W, y = (p / W) % H, z = p / (W * H);
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  return wrapi(x + dx, W) + W * (wrapi(y + dy, H) + H * wrapi(z + dz, D));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// out[p][co] = act(bias[co] + sum_{t, ci} w[co][t][ci] in[tap(p, t)][ci]).
// One warp: 16 consecutive positions x all C_out (NT = C_out/8 tiles of 8).
// A fragment (16 positions x 16 channels of one tap), B fragment (16
// channels x 8 output channels), C: FP32.
template <int NT>
__global__ void __launch_bounds__(128) k_conv_fwd(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias, float* __restrict__ out32,
                                                  __nv_bfloat16* __restrict__ out16, int npos, int W, int H, int D,
                                                  int cin, int taps, int relu) {
  constexpr int COUT = NT * 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p0 = (blockIdx.x * 4 + warp) * 16;
  if (p0 >= npos) return;
  const int g = lane >> 2, tg = lane & 3;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  const int pa = min(p0 + g, npos - 1), pb = min(p0 + g + 8, npos - 1);
  for (int t = 0; t < taps; ++t) {
    const int qa = tap_pos(pa, t, taps, W, H, D), qb = tap_pos(pb, t, taps, W, H, D);
    const __nv_bfloat16* ra = in + (size_t)qa * cin;
    const __nv_bfloat16* rb = in + (size_t)qb * cin;
    for (int c0 = 0; c0 < cin; c0 += 16) {
      uint32_t a[4];
      a[0] = ld2(ra + c0 + tg * 2);
      a[1] = ld2(rb + c0 + tg * 2);
      a[2] = ld2(ra + c0 + 8 + tg * 2);
      a[3] = ld2(rb + c0 + 8 + tg * 2);
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const __nv_bfloat16* wr = w + ((size_t)(j * 8 + g) * taps + t) * cin + c0;
        uint32_t b[2] = {ld2(wr + tg * 2), ld2(wr + 8 + tg * 2)};
        mma_bf16(acc[j], a, b);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int co = j * 8 + tg * 2;
    const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
    float v[4] = {acc[j][0] + b0, acc[j][1] + b1, acc[j][2] + b0, acc[j][3] + b1};
    if (relu)
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = fmaxf(v[k], 0.f);
    const int rows[2] = {p0 + g, p0 + g + 8};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (rows[r] >= npos) continue;
      const size_t o = (size_t)rows[r] * COUT + co;
      if (out32) {
        out32[o] = v[2 * r];
        out32[o + 1] = v[2 * r + 1];
      }
      if (out16) {
        out16[o] = __float2bfloat16_rn(v[2 * r]);
        out16[o + 1] = __float2bfloat16_rn(v[2 * r + 1]);
      }
    }
  }
}

// Partial dW[co][t][ci] = sum_p dout[p][co] in[tap(p, t)][ci] over one chunk
// of positions, stored for the chunk (part[chunk][co][t][ci]); one warp per
// (chunk, tap, 16 output channels).  A = dout^T (16 C_out x 16 positions),
// B = shifted input (16 positions x 8 C_in).
template <int NTI>
__global__ void __launch_bounds__(32) k_conv_wgrad(const __nv_bfloat16* __restrict__ dout,
                                                   const __nv_bfloat16* __restrict__ in, float* __restrict__ part,
                                                   int npos, int W, int H, int D, int cin, int cout, int taps,
                                                   int chunk) {
  const int lane = threadIdx.x, g = lane >> 2, tg = lane & 3;
  const int t = blockIdx.y, co0 = blockIdx.z * 16;
  const int pbeg = blockIdx.x * chunk, pend = min(npos, pbeg + chunk);
  float acc[NTI][4];
#pragma unroll
  for (int j = 0; j < NTI; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int p0 = pbeg; p0 < pend; p0 += 16) {
    // A[m = co][k = position]: a0 (g, 2tg..2tg+1), a1 (g+8, ...), a2 (g, 2tg+8..), a3 (g+8, 2tg+8..)
    int pk[4] = {p0 + tg * 2, p0 + tg * 2 + 1, p0 + tg * 2 + 8, p0 + tg * 2 + 9};
    __nv_bfloat16 da[4], db[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ok = pk[k] < pend;
      da[k] = ok ? dout[(size_t)pk[k] * cout + co0 + g] : zero;
      db[k] = ok ? dout[(size_t)pk[k] * cout + co0 + g + 8] : zero;
    }
    uint32_t a[4] = {pack2(da[0], da[1]), pack2(db[0], db[1]), pack2(da[2], da[3]), pack2(db[2], db[3])};
    int qk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) qk[k] = pk[k] < pend ? tap_pos(pk[k], t, taps, W, H, D) : -1;
#pragma unroll
    for (int j = 0; j < NTI; ++j) {
      // B[k = position][n = ci]: b0 rows 2tg, 2tg+1 col g; b1 rows 2tg+8, 2tg+9
      __nv_bfloat16 e[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) e[k] = qk[k] >= 0 ? in[(size_t)qk[k] * cin + j * 8 + g] : zero;
      uint32_t b[2] = {pack2(e[0], e[1]), pack2(e[2], e[3])};
      mma_bf16(acc[j], a, b);
    }
  }
  float* dw = part + (size_t)blockIdx.x * cout * taps * cin;
#pragma unroll
  for (int j = 0; j < NTI; ++j) {
    const int ci = j * 8 + tg * 2;
    dw[((size_t)(co0 + g) * taps + t) * cin + ci] = acc[j][0];
    dw[((size_t)(co0 + g) * taps + t) * cin + ci + 1] = acc[j][1];
    dw[((size_t)(co0 + g + 8) * taps + t) * cin + ci] = acc[j][2];
    dw[((size_t)(co0 + g + 8) * taps + t) * cin + ci + 1] = acc[j][3];
  }
}

// dw[e] += sum over the chunks, in chunk order, of part[chunk][e].
__global__ void k_wgrad_sum(const float* __restrict__ part, float* __restrict__ dw, int nchunk, size_t nw) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nw; e += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * nw + e];
    dw[e] += s;
  }
}

// Weights of the input-gradient convolution: w'[ci][t][co] = w[co][taps-1-t][ci].
__global__ void k_flip_weights(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt, int cout, int cin,
                               int taps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cout * cin * taps) return;
  const int co = i / (taps * cin), t = (i / cin) % taps, ci = i % cin;
  wt[((size_t)ci * taps + (taps - 1 - t)) * cout + co] = w[i];
}

__global__ void k_bias_grad(const float* __restrict__ dout, float* __restrict__ db, int npos, int c) {
  __shared__ float s[256];
  for (int ch = blockIdx.x; ch < c; ch += gridDim.x) {
    float v = 0.f;
    for (int p = threadIdx.x; p < npos; p += blockDim.x) v += dout[(size_t)p * c + ch];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
      if (threadIdx.x < d) s[threadIdx.x] += s[threadIdx.x + d];
      __syncthreads();
    }
    if (threadIdx.x == 0) db[ch] += s[0];
    __syncthreads();
  }
}

// dz = dy * (y > 0) (ReLU backward from the stored activation); also to BF16.
__global__ void k_relu_bwd(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ y, float* __restrict__ dz32,
                           __nv_bfloat16* __restrict__ dz16, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = __bfloat162float(y[i]) > 0.f ? dy[i] : 0.f;
    if (dz32) dz32[i] = v;
    if (dz16) dz16[i] = __float2bfloat16_rn(v);
  }
}

__global__ void k_cast_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// 2x2x2 mean pooling (channels last) and its adjoint.
__global__ void k_pool2(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out, int S, int c) {
  const int So = S / 2;
  const size_t n = (size_t)So * So * So * c;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    const size_t p = i / c;
    const int x = (int)(p % So), y = (int)((p / So) % So), z = (int)(p / ((size_t)So * So));
    float s = 0.f;
    for (int k = 0; k < 8; ++k) {
      const int xx = 2 * x + (k & 1), yy = 2 * y + ((k >> 1) & 1), zz = 2 * z + (k >> 2);
      s += __bfloat162float(in[((size_t)xx + (size_t)S * (yy + (size_t)S * zz)) * c + ch]);
    }
    out[i] = __float2bfloat16_rn(0.125f * s);
  }
}

__global__ void k_pool2_bwd(const float* __restrict__ dout, float* __restrict__ din, int S, int c) {
  const size_t n = (size_t)S * S * S * c;
  const int So = S / 2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    const size_t p = i / c;
    const int x = (int)(p % S), y = (int)((p / S) % S), z = (int)(p / ((size_t)S * S));
    din[i] += 0.125f * dout[((size_t)(x / 2) + (size_t)So * ((y / 2) + (size_t)So * (z / 2))) * c + ch];
  }
}

// Nearest x2 upsampling of a (So^3, c1) tensor into channels [0, c1) of a
// (2So)^3 tensor with c1 + c2 channels, and the copy of the skip tensor
// (c2 channels) into channels [c1, c1 + c2).
__global__ void k_up2_concat(const __nv_bfloat16* __restrict__ lo, const __nv_bfloat16* __restrict__ skip,
                             __nv_bfloat16* __restrict__ out, int S, int c1, int c2) {
  const int c = c1 + c2, So = S / 2;
  const size_t n = (size_t)S * S * S * c;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    const size_t p = i / c;
    if (ch < c1) {
      const int x = (int)(p % S), y = (int)((p / S) % S), z = (int)(p / ((size_t)S * S));
      out[i] = lo[((size_t)(x / 2) + (size_t)So * ((y / 2) + (size_t)So * (z / 2))) * c1 + ch];
    } else {
      out[i] = skip[p * c2 + (ch - c1)];
    }
  }
}

// Adjoint: d(lo) = sum of the 8 children of channels [0, c1); d(skip) += channels [c1, c).
__global__ void k_up2_concat_bwd(const float* __restrict__ dout, float* __restrict__ dlo, float* __restrict__ dskip,
                                 int S, int c1, int c2) {
  const int c = c1 + c2, So = S / 2;
  const size_t nlo = (size_t)So * So * So * c1;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nlo; i += (size_t)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c1);
    const size_t p = i / c1;
    const int x = (int)(p % So), y = (int)((p / So) % So), z = (int)(p / ((size_t)So * So));
    float s = 0.f;
    for (int k = 0; k < 8; ++k) {
      const int xx = 2 * x + (k & 1), yy = 2 * y + ((k >> 1) & 1), zz = 2 * z + (k >> 2);
      s += dout[((size_t)xx + (size_t)S * (yy + (size_t)S * zz)) * c + ch];
    }
    dlo[i] = s;
  }
  const size_t nsk = (size_t)S * S * S * c2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nsk; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / c2;
    dskip[i] += dout[p * c + c1 + (i % c2)];
  }
}

// Masked mean-square error over fluid positions and the 5 Q components of
// pred = base + out[:, 0:5] (out has cout channels); grad w.r.t. out.
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ base, const float* __restrict__ target,
                      const float* __restrict__ fluid, float* __restrict__ grad, double* __restrict__ loss, int npos,
                      int cout, double inv_count) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npos; p += gridDim.x * blockDim.x) {
    const float m = fluid[p];
    for (int c = 0; c < cout; ++c) {
      float gv = 0.f;
      if (c < 5 && m > 0.f) {
        const float d = out[(size_t)p * cout + c] + base[(size_t)p * 5 + c] - target[(size_t)p * 5 + c];
        acc += (double)d * d;
        gv = (float)(2.0 * inv_count) * d;
      }
      if (grad) grad[(size_t)p * cout + c] = gv;
    }
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int d = blockDim.x / 2; d > 0; d >>= 1) {
    if (threadIdx.x < d) s[threadIdx.x] += s[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, s[0] * inv_count);
}

// Cube means of the masked error (one thread per cube and component) and
// their squared sum; then each fluid position's share of the gradient.
__global__ void k_mse_coarse_blocks(const float* __restrict__ out, const float* __restrict__ base,
                                    const float* __restrict__ target, const float* __restrict__ fluid,
                                    float* __restrict__ blk, double* __restrict__ loss, int S, int b, int cout,
                                    double inv_count) {
  __shared__ double s[256];
  const int nc = S / b;
  const int ncube = nc * nc * nc;
  double acc = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncube * 5; t += gridDim.x * blockDim.x) {
    const int cube = t / 5, c = t % 5;
    const int cx = cube % nc, cy = (cube / nc) % nc, cz = cube / (nc * nc);
    double sum = 0.0;
    for (int dz = 0; dz < b; ++dz)
      for (int dy = 0; dy < b; ++dy)
        for (int dx = 0; dx < b; ++dx) {
          const size_t p = (size_t)(cx * b + dx) + (size_t)S * ((cy * b + dy) + (size_t)S * (cz * b + dz));
          if (fluid[p] > 0.f) sum += (double)(out[p * cout + c] + base[p * 5 + c] - target[p * 5 + c]);
        }
    const double e = sum / ((double)b * b * b);
    blk[t] = (float)e;
    acc += e * e;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int d = blockDim.x / 2; d > 0; d >>= 1) {
    if (threadIdx.x < d) s[threadIdx.x] += s[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, s[0] * inv_count);
}

__global__ void k_mse_coarse_grad(const float* __restrict__ fluid, const float* __restrict__ blk,
                                  float* __restrict__ grad, int S, int b, int cout, double inv_count) {
  const int nc = S / b;
  const size_t npos = (size_t)S * S * S;
  const float g = (float)(2.0 * inv_count / ((double)b * b * b));
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < npos; p += (size_t)gridDim.x * blockDim.x) {
    if (!(fluid[p] > 0.f)) continue;
    const int x = (int)(p % S), y = (int)((p / S) % S), z = (int)(p / ((size_t)S * S));
    const int cube = x / b + nc * (y / b + nc * (z / b));
    for (int c = 0; c < 5; ++c) grad[p * cout + c] += g * blk[cube * 5 + c];
  }
}

// Adam on FP32 masters with a BF16 working copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ p16, size_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (p16) p16[i] = __float2bfloat16_rn(pi);
  }
}

// Network input (channels last, cpad >= 9 channels, the rest zero):
// [solid indicator, Q xx,xy,xz,yy,yz, R/32, p/64, 20 w] from FP64 SoA fields.
__global__ void k_pack_input(const double* __restrict__ solid, const double* __restrict__ q, float r, float pitch,
                             float w, __nv_bfloat16* __restrict__ x16, float* __restrict__ base, float* __restrict__ fluid,
                             double* __restrict__ nfluid, int npos, int cpad) {
  int cnt = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npos; p += gridDim.x * blockDim.x) {
    cnt += solid[p] < 0.0;
    const bool sol = solid[p] >= 0.0;
    float v[9] = {sol ? 1.f : 0.f, 0, 0, 0, 0, 0, r / 32.f, pitch / 64.f, 20.f * w};
    for (int c = 0; c < 5; ++c) {
      v[1 + c] = (float)q[(size_t)c * npos + p];
      if (base) base[(size_t)p * 5 + c] = v[1 + c];
    }
    for (int c = 0; c < cpad; ++c) x16[(size_t)p * cpad + c] = __float2bfloat16_rn(c < 9 ? v[c] : 0.f);
    if (fluid) fluid[p] = sol ? 0.f : 1.f;
  }
  if (nfluid) {
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nfluid, (double)cnt);
  }
}

// SoA FP64 [5][npos] -> channels-last FP32 (npos x 5).
__global__ void k_from_soa(const double* __restrict__ q, float* __restrict__ a, int npos) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npos; p += gridDim.x * blockDim.x)
    for (int c = 0; c < 5; ++c) a[(size_t)p * 5 + c] = (float)q[(size_t)c * npos + p];
}

// Channels-last (npos, 5) FP32 -> SoA FP64 [5][npos].
__global__ void k_to_soa(const float* __restrict__ a, const float* __restrict__ base, double* __restrict__ q, int npos,
                         int cout) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npos; p += gridDim.x * blockDim.x)
    for (int c = 0; c < 5; ++c) q[(size_t)c * npos + p] = (double)a[(size_t)p * cout + c] + (base ? base[(size_t)p * 5 + c] : 0.0);
}

// Trilinear x2 upsampling of a periodic SoA field [c][S^3] (cell-centred: the
// fine node 2i + 1/2 +- 1/4 of coarse node i) to [c][(2S)^3].
__global__ void k_trilinear2(const double* __restrict__ a, double* __restrict__ b, int S, int c) {
  const int F = 2 * S;
  const size_t n = (size_t)F * F * F;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * c; i += (size_t)gridDim.x * blockDim.x) {
    const int ch = (int)(i / n);
    const size_t p = i % n;
    const int X = (int)(p % F), Y = (int)((p / F) % F), Z = (int)(p / ((size_t)F * F));
    int i0[3], i1[3];
    float t[3];
    const int P[3] = {X, Y, Z};
    for (int k = 0; k < 3; ++k) {
      // fine coordinate in coarse units: (P + 0.5)/2 - 0.5
      const float u = 0.5f * (P[k] + 0.5f) - 0.5f;
      const int f = (int)floorf(u);
      t[k] = u - f;
      i0[k] = wrapi(f, S);
      i1[k] = wrapi(f + 1, S);
    }
    double v = 0.0;
    for (int k = 0; k < 8; ++k) {
      const int xx = (k & 1) ? i1[0] : i0[0], yy = (k & 2) ? i1[1] : i0[1], zz = (k & 4) ? i1[2] : i0[2];
      const double wgt = ((k & 1) ? t[0] : 1 - t[0]) * ((k & 2) ? t[1] : 1 - t[1]) * ((k & 4) ? t[2] : 1 - t[2]);
      v += wgt * a[(size_t)ch * S * S * S + xx + (size_t)S * (yy + (size_t)S * zz)];
    }
    b[i] = v;
  }
}

static inline int grid_for(size_t n, int bs = 256) {
  size_t g = (n + bs - 1) / bs;
  return (int)(g > 65535 * 8 ? 65535 * 8 : (g < 1 ? 1 : g));
}

}  // namespace lcnn

using namespace lcnn;

extern "C" {

int lc_nn_conv3d_fwd(const void* in, const void* w, const float* bias, float* out32, void* out16, int W, int H, int D,
                     int cin, int cout, int taps, int relu, void* stream) {
  if (!in || !w || (!out32 && !out16) || cin % 16 || cout % 8 || cout > 80 || (taps != 27 && taps != 1) || W < 1 ||
      H < 1 || D < 1)
    return LC_NN_ERR_ARG;
  const int npos = W * H * D;
  const dim3 grid((npos + 63) / 64);
  cudaStream_t s = (cudaStream_t)stream;
  auto* a = (const __nv_bfloat16*)in;
  auto* b = (const __nv_bfloat16*)w;
  auto* o16 = (__nv_bfloat16*)out16;
  switch (cout / 8) {
    case 1: k_conv_fwd<1><<<grid, 128, 0, s>>>(a, b, bias, out32, o16, npos, W, H, D, cin, taps, relu); break;
    case 2: k_conv_fwd<2><<<grid, 128, 0, s>>>(a, b, bias, out32, o16, npos, W, H, D, cin, taps, relu); break;
    case 4: k_conv_fwd<4><<<grid, 128, 0, s>>>(a, b, bias, out32, o16, npos, W, H, D, cin, taps, relu); break;
    case 6: k_conv_fwd<6><<<grid, 128, 0, s>>>(a, b, bias, out32, o16, npos, W, H, D, cin, taps, relu); break;
    case 8: k_conv_fwd<8><<<grid, 128, 0, s>>>(a, b, bias, out32, o16, npos, W, H, D, cin, taps, relu); break;
    case 10: k_conv_fwd<10><<<grid, 128, 0, s>>>(a, b, bias, out32, o16, npos, W, H, D, cin, taps, relu); break;
    default: return LC_NN_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_conv3d_dgrad(const void* dout, const void* w, void* wt_scratch, float* din32, void* din16, int W, int H,
                       int D, int cin, int cout, int taps, void* stream) {
  if (!dout || !w || !wt_scratch || cout % 16 || cin % 8) return LC_NN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = cout * cin * taps;
  k_flip_weights<<<(n + 255) / 256, 256, 0, s>>>((const __nv_bfloat16*)w, (__nv_bfloat16*)wt_scratch, cout, cin, taps);
  if (cudaGetLastError() != cudaSuccess) return LC_NN_ERR_CUDA;
  return lc_nn_conv3d_fwd(dout, wt_scratch, nullptr, din32, din16, W, H, D, cout, cin, taps, 0, stream);
}

// Positions per chunk of the weight gradient: 1024, more when that would give
// more than 256 chunks (a multiple of 16, the MMA's K).
static int wgrad_chunk(int npos) {
  int chunk = 1024;
  while ((npos + chunk - 1) / chunk > 256) chunk *= 2;
  return chunk;
}

size_t lc_nn_wgrad_partial_floats(int W, int H, int D, int cin, int cout, int taps) {
  const int npos = W * H * D;
  if (npos <= 0) return 0;
  const int nchunk = (npos + wgrad_chunk(npos) - 1) / wgrad_chunk(npos);
  return (size_t)nchunk * cout * taps * cin;
}

int lc_nn_conv3d_wgrad(const void* dout, const void* in, float* dw, float* partial, int W, int H, int D, int cin,
                       int cout, int taps, void* stream) {
  if (!dout || !in || !dw || !partial || cout % 16 || cin % 8 || cin > 80) return LC_NN_ERR_ARG;
  const int npos = W * H * D;
  if (npos <= 0) return LC_NN_ERR_ARG;
  const int chunk = wgrad_chunk(npos);
  const int nchunk = (npos + chunk - 1) / chunk;
  const dim3 grid(nchunk, taps, cout / 16);
  cudaStream_t s = (cudaStream_t)stream;
  auto* a = (const __nv_bfloat16*)dout;
  auto* b = (const __nv_bfloat16*)in;
  switch (cin / 8) {
    case 1: k_conv_wgrad<1><<<grid, 32, 0, s>>>(a, b, partial, npos, W, H, D, cin, cout, taps, chunk); break;
    case 2: k_conv_wgrad<2><<<grid, 32, 0, s>>>(a, b, partial, npos, W, H, D, cin, cout, taps, chunk); break;
    case 4: k_conv_wgrad<4><<<grid, 32, 0, s>>>(a, b, partial, npos, W, H, D, cin, cout, taps, chunk); break;
    case 6: k_conv_wgrad<6><<<grid, 32, 0, s>>>(a, b, partial, npos, W, H, D, cin, cout, taps, chunk); break;
    case 10: k_conv_wgrad<10><<<grid, 32, 0, s>>>(a, b, partial, npos, W, H, D, cin, cout, taps, chunk); break;
    default: return LC_NN_ERR_ARG;
  }
  const size_t nw = (size_t)cout * taps * cin;
  k_wgrad_sum<<<grid_for(nw), 256, 0, s>>>(partial, dw, nchunk, nw);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_bias_grad(const float* dout, float* db, int npos, int c, void* stream) {
  k_bias_grad<<<c, 256, 0, (cudaStream_t)stream>>>(dout, db, npos, c);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_relu_bwd(const float* dy, const void* y, float* dz32, void* dz16, size_t n, void* stream) {
  k_relu_bwd<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(dy, (const __nv_bfloat16*)y, dz32, (__nv_bfloat16*)dz16, n);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_cast_bf16(const float* a, void* b, size_t n, void* stream) {
  k_cast_bf16<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(a, (__nv_bfloat16*)b, n);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_pool2(const void* in, void* out, int S, int c, void* stream) {
  if (S % 2) return LC_NN_ERR_ARG;
  k_pool2<<<grid_for((size_t)S * S * S * c / 8), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)in,
                                                                                   (__nv_bfloat16*)out, S, c);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_pool2_bwd(const float* dout, float* din, int S, int c, void* stream) {
  k_pool2_bwd<<<grid_for((size_t)S * S * S * c), 256, 0, (cudaStream_t)stream>>>(dout, din, S, c);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_up2_concat(const void* lo, const void* skip, void* out, int S, int c1, int c2, void* stream) {
  if (S % 2) return LC_NN_ERR_ARG;
  k_up2_concat<<<grid_for((size_t)S * S * S * (c1 + c2)), 256, 0, (cudaStream_t)stream>>>(
      (const __nv_bfloat16*)lo, (const __nv_bfloat16*)skip, (__nv_bfloat16*)out, S, c1, c2);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_up2_concat_bwd(const float* dout, float* dlo, float* dskip, int S, int c1, int c2, void* stream) {
  k_up2_concat_bwd<<<grid_for((size_t)S * S * S * c2), 256, 0, (cudaStream_t)stream>>>(dout, dlo, dskip, S, c1, c2);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_mse(const float* out, const float* base, const float* target, const float* fluid, float* grad,
              double* loss, int npos, int cout, double inv_count, void* stream) {
  k_mse<<<grid_for(npos), 256, 0, (cudaStream_t)stream>>>(out, base, target, fluid, grad, loss, npos, cout, inv_count);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_mse_coarse(const float* out, const float* base, const float* target, const float* fluid, float* grad,
                     double* loss, float* blk, int S, int b, int cout, double inv_count, void* stream) {
  if (b < 1 || S < 1 || S % b != 0 || cout < 5 || !blk || !loss) return LC_NN_ERR_ARG;
  const int nc = S / b;
  cudaStream_t st = (cudaStream_t)stream;
  k_mse_coarse_blocks<<<grid_for((size_t)nc * nc * nc * 5), 256, 0, st>>>(out, base, target, fluid, blk, loss, S, b,
                                                                           cout, inv_count);
  if (grad) k_mse_coarse_grad<<<grid_for((size_t)S * S * S), 256, 0, st>>>(fluid, blk, grad, S, b, cout, inv_count);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_adam(float* p, const float* g, float* m, float* v, void* p16, size_t n, float lr, float b1, float b2,
               float eps, int step, void* stream) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, (__nv_bfloat16*)p16, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_pack_input(const double* solid, const double* q, double R, double pitch, double w, void* x16, float* base,
                     float* fluid, double* nfluid, int npos, int cpad, void* stream) {
  if (cpad < 9) return LC_NN_ERR_ARG;
  k_pack_input<<<grid_for(npos), 256, 0, (cudaStream_t)stream>>>(solid, q, (float)R, (float)pitch, (float)w,
                                                                   (__nv_bfloat16*)x16, base, fluid, nfluid, npos, cpad);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_from_soa(const double* q, float* a, int npos, void* stream) {
  k_from_soa<<<grid_for(npos), 256, 0, (cudaStream_t)stream>>>(q, a, npos);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_to_soa(const float* a, const float* base, double* q, int npos, int cout, void* stream) {
  k_to_soa<<<grid_for(npos), 256, 0, (cudaStream_t)stream>>>(a, base, q, npos, cout);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

int lc_nn_trilinear2(const double* a, double* b, int S, int c, void* stream) {
  k_trilinear2<<<grid_for((size_t)8 * S * S * S * c), 256, 0, (cudaStream_t)stream>>>(a, b, S, c);
  return cudaGetLastError() == cudaSuccess ? LC_NN_OK : LC_NN_ERR_CUDA;
}

}  // extern "C"
