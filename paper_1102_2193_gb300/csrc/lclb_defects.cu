// lclb_defects.cu -- defect analytics of one box (Sec. 3.1, 3.2).
//
// A defect node is a fluid node whose scalar order 3/2 lambda_max(Q) is below
// a threshold (0.435 in the paper, the isosurface level of its defect
// renderings); the disclination loops of Sec. 3.2 (Saturn ring, figure of
// eight) and the boojums of Sec. 3.1 are the connected sets of such nodes.
//   k_def_init     defect test per node (FP64 from the stored Q, by Sylvester's
//                  criterion), parent[i] = i or -1
//   k_def_union    union-find over the +x, +y, +z face links between defect nodes
//                  (lock-free: a root is linked under the smaller root by CAS, so
//                  the root of every set is its smallest node index)
//   k_def_flatten  parent[i] = root of i
//   k_def_count / k_def_scan / k_def_rank
//                  components numbered in root order (block counts, one-block
//                  exclusive scan, in-block ranks)
//   k_def_sum1 / k_def_centroid / k_def_sum2 / k_def_final
//                  node count, periodic (circular-mean) centroid, gyration tensor
//                  of the minimum-image displacements, FP64 sums
// Every find and union loop is bounded; a loop that reaches its bound sets
// an error flag that the host reads (it cannot happen: every link points to a
// smaller index, so each loop strictly descends).
#include "lclb_dev.cuh"
#include "lclb_internal.h"

namespace lclb {

constexpr int DEF_ITER_MAX = 1 << 24;
constexpr double DEF_TWO_PI = 6.283185307179586476925286766559;

// Defect test 3/2 lambda_max(Q) < thr without the eigenvalue: with
// t = thr / 1.5, every eigenvalue of the symmetric Q is below t exactly when
// t I - Q is positive definite, i.e. (Sylvester's criterion) when its three
// leading principal minors are positive.  FP64 multiply-adds only.
__device__ __forceinline__ bool def_is_defect(const double q[5], double t) {
  const double m00 = t - q[0], m11 = t - q[3], m22 = t + q[0] + q[3];
  const double m01 = -q[1], m02 = -q[2], m12 = -q[4];
  if (!(m00 > 0.0) || !(m00 * m11 - m01 * m01 > 0.0)) return false;
  return m00 * (m11 * m22 - m12 * m12) - m01 * (m01 * m22 - m12 * m02) + m02 * (m01 * m12 - m11 * m02) > 0.0;
}

// Root of x.  parent values only ever point to smaller indices, so x
// strictly decreases.  While the unions run, path halving (HALVE) stores a
// grandparent, an ancestor, on the way.  The flattening pass must not halve:
// a halving store from one thread could overwrite the root that another
// thread has just written for its own node.
template <bool HALVE>
__device__ __forceinline__ int def_find(int* parent, int x, int* err) {
  volatile int* vp = parent;
  for (int it = 0; it < DEF_ITER_MAX; ++it) {
    const int p = vp[x];
    if (p == x) return x;
    if (HALVE) {
      const int gp = vp[p];
      if (gp != p) vp[x] = gp;
      x = gp;
    } else {
      x = p;
    }
  }
  atomicExch(err, 1);
  return x;
}

__device__ __forceinline__ void def_union(int* parent, int a, int b, int* err) {
  for (int it = 0; it < DEF_ITER_MAX; ++it) {
    a = def_find<true>(parent, a, err);
    b = def_find<true>(parent, b, err);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(parent + a, a, b) == a) return;  // else a was linked meanwhile: retry
  }
  atomicExch(err, 1);
}

template <typename T>
__global__ void __launch_bounds__(256) k_def_init(const DevBox* __restrict__ boxes, int b, double thr,
                                                  int* __restrict__ parent) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N) return;
  int v = -1;
  if ((B.mask[i] & IDMASK) == 0) {
    double q[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) q[k] = load_q<T>(B, i, k);
    if (def_is_defect(q, thr / 1.5)) v = i;
  }
  parent[i] = v;
}

__global__ void __launch_bounds__(256) k_def_union(const DevBox* __restrict__ boxes, int b, int* parent, int* err) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N || parent[i] < 0) return;
  const int nx = B.nx, ny = B.ny, nz = B.nz;
  const int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
  const int js[3] = {(x + 1 == nx ? 0 : x + 1) + nx * (y + ny * z), x + nx * ((y + 1 == ny ? 0 : y + 1) + ny * z),
                     (B.wall_z && z + 1 == nz) ? -1 : x + nx * (y + ny * (z + 1 == nz ? 0 : z + 1))};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int j = js[d];
    if (j >= 0 && j != i && parent[j] >= 0) def_union(parent, i, j, err);
  }
}

__global__ void __launch_bounds__(256) k_def_flatten(int N, int* parent, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || parent[i] < 0) return;
  parent[i] = def_find<false>(parent, i, err);
}

// Roots (parent[i] == i) per block of 256 nodes.
__global__ void __launch_bounds__(256) k_def_count(int N, const int* __restrict__ parent, int* __restrict__ blockcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool root = i < N && parent[i] == i;
  const int c = __syncthreads_count(root);
  if (threadIdx.x == 0) blockcnt[blockIdx.x] = c;
}

// Exclusive scan of nb block counts in place (one block); total -> *total.
__global__ void __launch_bounds__(1024) k_def_scan(int* a, int nb, int* total) {
  __shared__ int s[1024];
  const int t = threadIdx.x;
  const int per = (nb + 1023) / 1024;
  const int lo = min(nb, t * per), hi = min(nb, lo + per);
  int sum = 0;
  for (int k = lo; k < hi; ++k) sum += a[k];
  s[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = t >= off ? s[t - off] : 0;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  int run = s[t] - sum;  // exclusive prefix of this thread's range
  for (int k = lo; k < hi; ++k) {
    const int v = a[k];
    a[k] = run;
    run += v;
  }
  if (t == 1023) *total = s[1023];
}

// Component number of each root, in root order: comp[root] = its rank; list[rank] = root.
__global__ void __launch_bounds__(256) k_def_rank(int N, const int* __restrict__ parent,
                                                  const int* __restrict__ blockoff, int* __restrict__ comp,
                                                  int* __restrict__ list) {
  __shared__ int wsum[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool root = i < N && parent[i] == i;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, root);
  if (lane == 0) wsum[w] = __popc(m);
  __syncthreads();
  int off = blockoff[blockIdx.x];
  for (int k = 0; k < w; ++k) off += wsum[k];
  if (root) {
    const int r = off + __popc(m & ((1u << lane) - 1u));
    comp[i] = r;
    list[r] = i;
  }
}

// Node counts and the sums of the periodic centroid: per component c,
// circ[6c + 2a] += cos(2 pi x_a / L_a), circ[6c + 2a + 1] += sin(...), or for
// a walled z axis circ[6c + 4] += z.
__global__ void __launch_bounds__(256) k_def_sum1(const DevBox* __restrict__ boxes, int b,
                                                  const int* __restrict__ parent, const int* __restrict__ comp,
                                                  int* __restrict__ size, double* __restrict__ circ) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N || parent[i] < 0) return;
  const int c = comp[parent[i]];
  const int nx = B.nx, ny = B.ny, nz = B.nz;
  const int co[3] = {i % nx, (i / nx) % ny, i / (nx * ny)};
  const int L[3] = {nx, ny, nz};
  atomicAdd(size + c, 1);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == 2 && B.wall_z) {
      atomicAdd(circ + 6 * c + 4, (double)co[2]);
      continue;
    }
    const double th = DEF_TWO_PI * (double)co[a] / (double)L[a];
    atomicAdd(circ + 6 * c + 2 * a, cos(th));
    atomicAdd(circ + 6 * c + 2 * a + 1, sin(th));
  }
}

// Centroid of each component: the circular mean angle times L / 2 pi, moved
// into [0, L) (shifted by L when negative, taken back by L when that rounds
// to L); the plain mean along a walled z axis.
__global__ void k_def_centroid(const DevBox* __restrict__ boxes, int b, int ncomp, const int* __restrict__ size,
                               const double* __restrict__ circ, double* __restrict__ cen) {
  const DevBox& B = boxes[b];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncomp) return;
  const double n = (double)size[c];
  const int L[3] = {B.nx, B.ny, B.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == 2 && B.wall_z) {
      cen[3 * c + 2] = circ[6 * c + 4] / n;
      continue;
    }
    const double La = (double)L[a];
    double v = atan2(circ[6 * c + 2 * a + 1] / n, circ[6 * c + 2 * a] / n) * La / DEF_TWO_PI;
    if (v < 0.0) v += La;
    if (v >= La) v -= La;
    cen[3 * c + a] = v;
  }
}

// Sums of d_a d_b, d the minimum-image displacement of the node from its
// component's centroid (each periodic component wrapped into [-L/2, L/2)).
__global__ void __launch_bounds__(256) k_def_sum2(const DevBox* __restrict__ boxes, int b,
                                                  const int* __restrict__ parent, const int* __restrict__ comp,
                                                  const double* __restrict__ cen, double* __restrict__ gyr) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N || parent[i] < 0) return;
  const int c = comp[parent[i]];
  const int nx = B.nx, ny = B.ny, nz = B.nz;
  const int co[3] = {i % nx, (i / nx) % ny, i / (nx * ny)};
  const int L[3] = {nx, ny, nz};
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d[a] = (double)co[a] - cen[3 * c + a];
    if (!(a == 2 && B.wall_z)) d[a] = d[a] - (double)L[a] * floor(d[a] / (double)L[a] + 0.5);
  }
  atomicAdd(gyr + 6 * c + 0, d[0] * d[0]);
  atomicAdd(gyr + 6 * c + 1, d[0] * d[1]);
  atomicAdd(gyr + 6 * c + 2, d[0] * d[2]);
  atomicAdd(gyr + 6 * c + 3, d[1] * d[1]);
  atomicAdd(gyr + 6 * c + 4, d[1] * d[2]);
  atomicAdd(gyr + 6 * c + 5, d[2] * d[2]);
}

__global__ void k_def_final(int ncomp, const int* __restrict__ size, double* __restrict__ gyr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 6 * ncomp) return;
  gyr[k] /= (double)size[k / 6];
}

static inline int def_blocks(int n, int bs) { return (n + bs - 1) / bs; }

int defect_blocks(int N) { return def_blocks(N, 256); }

cudaError_t launch_defects_label(int prec, const DevBox* boxes, int b, int N, double thr, int* parent, int* comp,
                                 int* list, int* blockcnt, int* total, int* err, cudaStream_t s) {
  const int nb = def_blocks(N, 256);
  if (prec == 0) k_def_init<float><<<nb, 256, 0, s>>>(boxes, b, thr, parent);
  else k_def_init<double><<<nb, 256, 0, s>>>(boxes, b, thr, parent);
  k_def_union<<<nb, 256, 0, s>>>(boxes, b, parent, err);
  k_def_flatten<<<nb, 256, 0, s>>>(N, parent, err);
  k_def_count<<<nb, 256, 0, s>>>(N, parent, blockcnt);
  k_def_scan<<<1, 1024, 0, s>>>(blockcnt, nb, total);
  k_def_rank<<<nb, 256, 0, s>>>(N, parent, blockcnt, comp, list);
  return cudaGetLastError();
}

cudaError_t launch_defects_stats(const DevBox* boxes, int b, int N, int ncomp, const int* parent, const int* comp,
                                 int* size, double* circ, double* cen, double* gyr, cudaStream_t s) {
  if (ncomp <= 0) return cudaSuccess;
  const int nb = def_blocks(N, 256);
  k_def_sum1<<<nb, 256, 0, s>>>(boxes, b, parent, comp, size, circ);
  k_def_centroid<<<def_blocks(ncomp, 128), 128, 0, s>>>(boxes, b, ncomp, size, circ, cen);
  k_def_sum2<<<nb, 256, 0, s>>>(boxes, b, parent, comp, cen, gyr);
  k_def_final<<<def_blocks(6 * ncomp, 256), 256, 0, s>>>(ncomp, size, gyr);
  return cudaGetLastError();
}

}  // namespace lclb
