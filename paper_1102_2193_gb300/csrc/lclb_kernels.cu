// lclb_kernels.cu -- sm_103a kernels of one coupled step (Lintuvuori et al., Sec. 2.2):
//   k_force   LC stress at fluid nodes, its face divergence (body force) and the
//             colloid LC force/torque (Eqs. 4, 8); z-marching tiles with the
//             stress of three planes in shared memory.
//   k_lb      pull-scheme stream + BGK collide with Guo forcing, bounce-back on
//             links inline (moving-surface term), writes df* and u.
//   k_lc      Beris-Edwards update of Q (Eq. 2 with co-rotation and upwind
//             advective face fluxes), residual partials.
//   k_links   momentum exchange over the boundary-link list -> F_hyd, T_hyd.
//   k_colloid colloid update and buffer-parity flip.
// All step kernels walk a work list of (box, x0, y0, z0) tiles, so that one
// launch serves one box or a batch of boxes of different sizes.
#include <cstdio>

#include "lclb_dev.cuh"
#include "lclb_f2.cuh"
#include "lclb_internal.h"

namespace lclb {

constexpr int TX = 32;

// Loads of data that the same launch may have written (the persistent step
// kernel: stress, velocity, post-collision populations, colloid sums) go
// through L2 only (CG); data produced by earlier launches may take the
// read-only path.
template <bool CG, typename T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}

// L2 eviction priorities (PTX createpolicy, cache hints on the loads and
// stores; no setting of the device changes): the stress, molecular field and
// velocity that the next kernels of the step read are stored to stay
// (evict_last), the populations, read and written once per step, to go first
// (evict_first), so the 129 MB L2 keeps the intermediates between kernels.
__device__ __forceinline__ uint64_t l2_keep() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_stream() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_hint(float* a, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(double* a, double v, uint64_t) { *a = v; }
__device__ __forceinline__ float ld_hint(const float* a, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_hint(const double* a, uint64_t) { return __ldg(a); }

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block sum of NV doubles per thread; result valid in thread 0.  sred needs
// 32*NV doubles.  Must be called by all threads of the block.
template <int NV>
__device__ void block_sum(double v[NV], double* sred, bool is_max_last = false) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = (is_max_last && k == NV - 1) ? warp_max(v[k]) : warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sred[k * 32 + wid] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sred[k * 32 + lane] : 0.0;
      v[k] = (is_max_last && k == NV - 1) ? warp_max(t) : warp_sum(t);
    }
  }
  __syncthreads();
}

// Residual partials of a warp's row of a Q-update tile: the sum of squares
// and the max over its lanes, written by lane 0 to part[2 wy], part[2 wy + 1]
// (one record per warp, so a tile needs no block barrier and no FP64 sum).
template <typename T>
__device__ __forceinline__ void warp_residual(double* part, int wy, int lane, T rsum, T rmax) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rsum += __shfl_down_sync(0xffffffffu, rsum, o);
    const T m = __shfl_down_sync(0xffffffffu, rmax, o);
    rmax = m > rmax ? m : rmax;
  }
  if (lane == 0) {
    part[2 * wy] = (double)rsum;
    part[2 * wy + 1] = (double)rmax;
  }
}

// Add per-lane contributions v[0..5] (for colloid id c, -1: none) into
// acc[off..off+NV-1] of each colloid with one FP64 atomic per (warp, colloid,
// component).  Must be called by all 32 lanes of a converged warp.
template <int NV = 6>
__device__ __forceinline__ void warp_flush_colloid(DevColloid* col, int c, const double* v, int off) {
  unsigned pend = __ballot_sync(0xffffffffu, c >= 0);
  const int lane = threadIdx.x & 31;
  while (pend) {
    const int leader = __ffs(pend) - 1;
    const int cc = __shfl_sync(0xffffffffu, c, leader);
    const bool mine = (c == cc);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double t = warp_sum(mine ? v[k] : 0.0);  // total lands in lane 0
      if (lane == 0 && t != 0.0) atomicAdd(&col[cc].acc[off + k], t);
    }
    if (mine) c = -1;
    pend = __ballot_sync(0xffffffffu, c >= 0);
  }
}

// The block's shared copy of box b's record, copied by all threads in 4-byte
// words (DevBox is a multiple of 8 bytes and 8-byte aligned).
static_assert(sizeof(DevBox) % 4 == 0, "DevBox is copied in 4-byte words");
__device__ __forceinline__ void load_box(DevBox& sb, const DevBox* boxes, int b) {
  __syncthreads();
  const unsigned* src = reinterpret_cast<const unsigned*>(boxes + b);
  unsigned* dst = reinterpret_cast<unsigned*>(&sb);
  const int nthr = blockDim.x * blockDim.y;
  for (int k = threadIdx.x + blockDim.x * threadIdx.y; k < (int)(sizeof(DevBox) / 4); k += nthr) dst[k] = src[k];
  __syncthreads();
}

// Tile loops: reload the shared box record only when the tile's box changes
// (b is uniform over the block, so the barriers are too).
__device__ __forceinline__ void load_box(DevBox& sb, const DevBox* boxes, int b, int& cur) {
  if (b == cur) return;
  load_box(sb, boxes, b);
  cur = b;
}

// ---------------------------------------------------------------------------
// shared pieces of the force / LB kernels
// ---------------------------------------------------------------------------
// Stress P (9 comps) of fluid node (gx,gy,kk) into sP[c*HP] (c = 0..8); the
// node's mask byte decides fluid/solid.  Returns the flag stored with it:
// 0 fluid, colloid id + 1, or WALLFLAG.  When hout is non-null (an interior
// position of the tile) the molecular field H is also stored there, for the
// Q update of the same step.
template <typename T>
__device__ __forceinline__ uint8_t stress_at(const DevBox& B, const PhysT<T>& PP, const T* __restrict__ Q, int gx,
                                             int gy, int kk, T* sP, int HP, bool fe, double* fe_acc, T* hout) {
  const int i = gx + B.nx * (gy + B.ny * kk);
  const uint8_t m = B.mask[i];
  const uint8_t flag = m & IDMASK;
  if (flag != 0) return flag;
  T qi[5], qn[6][5], h[5], p[9], fp;
  double surf = 0.0;
  gather_q(B, Q, gx, gy, kk, i, m, qi, qn, fe ? &surf : nullptr);
  lc_node<T, true>(PP, qi, qn, h, p, &fp);
#pragma unroll
  for (int c = 0; c < 9; ++c) sP[c * HP] = p[c];
  if (hout) {
#pragma unroll
    for (int c = 0; c < 5; ++c) hout[(size_t)c * B.N + i] = h[c];
  }
  if (fe) *fe_acc += (double)fp + surf;
  return 0;
}

// Colloid c takes -sgn P_{.,ax}(i) through the face of fluid node (x, y, kc)
// on its side (Eq. 8), with the moment about its centre; summed per thread
// into my_acc (F, T) for colloid my_c.
template <typename T>
__device__ __forceinline__ void colloid_face(const DevBox& B, int c, int ax, T sgn, const T pcv[3], int x, int y,
                                             int kc, int& my_c, double my_acc[6]) {
  const DevColloid& C = B.col[c];
  const T ff[3] = {-sgn * pcv[0], -sgn * pcv[1], -sgn * pcv[2]};
  double rd[3];
  const double hx2 = 0.5 * (double)(ax == 0 ? sgn : 0), hy2 = 0.5 * (double)(ax == 1 ? sgn : 0),
               hz2 = 0.5 * (double)(ax == 2 ? sgn : 0);
  disp(B, (double)x + hx2, (double)y + hy2, (double)kc + hz2, C.X, rd);
  // the face force is in T; its moment arm from the FP64 offset, taken in T
  const T r[3] = {T(rd[0]), T(rd[1]), T(rd[2])};
  const T tq[3] = {r[1] * ff[2] - r[2] * ff[1], r[2] * ff[0] - r[0] * ff[2], r[0] * ff[1] - r[1] * ff[0]};
  if (my_c >= 0 && my_c != c) {  // a second colloid at this node: flush the first directly
    for (int a = 0; a < 6; ++a) {
      atomicAdd(&B.col[my_c].acc[6 + a], my_acc[a]);
      my_acc[a] = 0.0;
    }
  }
  my_c = c;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    my_acc[a] += (double)ff[a];
    my_acc[3 + a] += (double)tq[a];
  }
}

// Body force at interior fluid position pc (plane slot s0; the planes below
// and above in slots sm, sp): F_a = sum_d [P_ad(face +d) - P_ad(face -d)],
// a fluid-fluid face carrying (P_i + P_j)/2 and a solid or wall face P_i.
// Each colloid face adds -(+-P_.d(i)) to the colloid's LC force (and its
// moment about X to the torque) in the thread's accumulator.
template <typename T>
__device__ __forceinline__ void face_force(const DevBox& B, const T* sP, const uint8_t* sFl, int HP, int HX, int s0,
                                           int sm, int sp, int pc, int x, int y, int kc, bool acc, T Fv[3],
                                           int& my_c, double my_acc[6]) {
  Fv[0] = Fv[1] = Fv[2] = T(0);
  const int nslot[6] = {s0, s0, s0, s0, sp, sm};
  const int npos[6] = {pc + 1, pc - 1, pc + HX, pc - HX, pc, pc};
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int ax = d >> 1;
    const T sgn = (d & 1) ? T(-1) : T(1);
    const uint8_t fj = sFl[nslot[d] * HP + npos[d]];
    T pcv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      pcv[a] = sP[(s0 * 9 + 3 * a + ax) * HP + pc];
      const T face = (fj == 0) ? T(0.5) * (pcv[a] + sP[(nslot[d] * 9 + 3 * a + ax) * HP + npos[d]]) : pcv[a];
      Fv[a] += sgn * face;
    }
    if (acc && fj != 0 && fj != WALLFLAG) colloid_face(B, fj - 1, ax, sgn, pcv, x, y, kc, my_c, my_acc);
  }
}

// ---------------------------------------------------------------------------
// k_force: body force (and, in diagnostic mode, free-energy partials) alone
// ---------------------------------------------------------------------------
// Shared memory: P of three z planes over the tile plus a one-node halo,
// [3][9][(TX+2)(TY+2)] in T, then one flag byte per position.
template <typename T, int TY>
__global__ void __launch_bounds__(TX * TY) k_force(const DevBox* __restrict__ boxes, const int4* __restrict__ tiles,
                                                   int ntiles, int zc, int mode, double* __restrict__ part) {
  constexpr int HX = TX + 2, HY = TY + 2, HP = HX * HY, NT = TX * TY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sP = reinterpret_cast<T*>(smem_raw);
  uint8_t* sFl = smem_raw + sizeof(T) * 27 * HP;
  __shared__ DevBox B;
  __shared__ double sred[32 * 1];
  const int tid = threadIdx.x + TX * threadIdx.y;

  int cur_box = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = tiles[t];
    load_box(B, boxes, td.x, cur_box);
    if (!B.p.lc_on) continue;
    const PhysT<T>& PP = phys<T>(B);
    int my_c = -1;
    double my_acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const T* __restrict__ Q = static_cast<const T*>(B.Q[B.st->qpar]);
    T* __restrict__ Fout = static_cast<T*>(B.F);
    const int x0 = td.y, y0 = td.z, z0 = td.w;
    const int nx = B.nx, ny = B.ny, nz = B.nz, N = B.N;
    const int vx = min(TX, nx - x0), vy = min(TY, ny - y0);
    const int zend = min(z0 + zc, nz);
    double fe_acc = 0.0;
    __syncthreads();
    for (int k = z0 - 1; k <= zend; ++k) {
      const int slot = (k - z0 + 1) % 3;
      const bool wallplane = B.wall_z && (k < 0 || k >= nz);
      const int kk = B.wall_z ? k : wrapn(k, nz);
      for (int pidx = tid; pidx < HP; pidx += NT) {
        const int hx = pidx % HX, hy = pidx / HX;
        if (hx > vx + 1 || hy > vy + 1) continue;
        uint8_t flag = WALLFLAG;
        if (!wallplane) {
          const bool inner = hx >= 1 && hx <= vx && hy >= 1 && hy <= vy && k >= z0 && k < zend;
          flag = stress_at(B, PP, Q, wrapn(x0 - 1 + hx, nx), wrapn(y0 - 1 + hy, ny), kk, sP + slot * 9 * HP + pidx,
                           HP, inner && (mode & FORCE_FE), &fe_acc, inner ? static_cast<T*>(B.H) : (T*)nullptr);
        }
        sFl[slot * HP + pidx] = flag;
      }
      __syncthreads();
      if (k >= z0 + 1) {
        const int kc = k - 1;
        const int tx = threadIdx.x, ty = threadIdx.y;
        const int pc = (tx + 1) + HX * (ty + 1);
        if (tx < vx && ty < vy && sFl[((k - z0) % 3) * HP + pc] == 0) {
          T Fv[3];
          face_force(B, sP, sFl, HP, HX, (k - z0) % 3, (k - z0 - 1) % 3, slot, pc, x0 + tx, y0 + ty, kc,
                     (mode & FORCE_ACC) != 0, Fv, my_c, my_acc);
          const int ic = (x0 + tx) + nx * ((y0 + ty) + ny * kc);
#pragma unroll
          for (int a = 0; a < 3; ++a) Fout[(size_t)a * N + ic] = Fv[a];
        }
      }
      __syncthreads();
    }
    if (mode & FORCE_ACC) warp_flush_colloid(B.col, my_c, my_acc, 6);
    if (mode & FORCE_FE) {
      double v[1] = {fe_acc};
      block_sum<1>(v, sred);
      if (tid == 0) part[t] = v[0];
    }
  }
}

// ---------------------------------------------------------------------------
// pull with bounce-back (shared by the LB kernels and the export/diagnostic kernels)
// ---------------------------------------------------------------------------
// Gathers the pre-collision deviations df_q(r) = df*_q(r - c_q) for fluid
// node r, or, when r - c_q is solid (colloid) or beyond a wall, the bounced
// population df*_{-q}(r) + 6 w_q rho0 (c_q . u_b) with u_b the rigid velocity
// at the link midpoint r - c_q/2 of the state that produced df* (Vb, Wb, Xb).
template <typename T>
__device__ __forceinline__ void pull(const DevBox& B, const T* __restrict__ fin, int x, int y, int z, int i, uint8_t m,
                                     bool pre, T df[NQ]) {
  const int N = B.N;
  if (pre) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) df[q] = ldg(fin + (size_t)q * N + i);
    return;
  }
  const int nx = B.nx, ny = B.ny, nz = B.nz;
  const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x + 1 == nx ? 0 : x + 1};
  const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y + 1 == ny ? 0 : y + 1};
  int zs[3];
  if (B.wall_z) {
    zs[0] = z - 1; zs[1] = z; zs[2] = z + 1;
  } else {
    zs[0] = z == 0 ? nz - 1 : z - 1; zs[1] = z; zs[2] = z + 1 == nz ? 0 : z + 1;
  }
  if (!(m & NEAR)) {
    const uint64_t pol = l2_stream();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int s = xs[1 - cx(q)] + nx * (ys[1 - cy(q)] + ny * zs[1 - cz(q)]);
      df[q] = ld_hint(fin + (size_t)q * N + s, pol);
    }
    return;
  }
  const T rho0 = phys<T>(B).rho0;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int zsrc = zs[1 - cz(q)];
    int s = -1;
    uint8_t ms = WALLFLAG;
    if (zsrc >= 0 && zsrc < nz) {
      s = xs[1 - cx(q)] + nx * (ys[1 - cy(q)] + ny * zsrc);
      ms = B.mask[s] & IDMASK;
    }
    if (ms == 0) {
      df[q] = ldg(fin + (size_t)q * N + s);
    } else {
      T corr = T(0);
      if (ms != WALLFLAG) {
        const DevColloid& C = B.col[ms - 1];
        T ub[3];
        rigid_velocity_t<T>(B, T(x) - T(0.5 * cx(q)), T(y) - T(0.5 * cy(q)), T(z) - T(0.5 * cz(q)), C.Xb, C.Vb, C.Wb,
                            ub);
        const T cub = T(cx(q)) * ub[0] + T(cy(q)) * ub[1] + T(cz(q)) * ub[2];
        corr = T(6.0 * wq(q)) * rho0 * cub;
      }
      df[q] = ldg(fin + (size_t)opp(q) * N + i) + corr;
    }
  }
}

// Collide at fluid node i with force (Fx,Fy,Fz) (BGK + Guo, deviation form):
// rho = rho0 + sum df, u = (sum df c + F/2)/rho,
// df*_q = df_q - omega (df_q - df_eq_q) + (1 - 1/2tau) w_q [3(c - u) + 9 (c.u) c].F,
// df_eq_q = w_q [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)].  Writes df* and u.
template <typename T>
__device__ __forceinline__ void collide_store(const PhysT<T>& PP, T* __restrict__ fout, T* __restrict__ ub, int N,
                                              int i, const T df[NQ], T Fx, T Fy, T Fz) {
  T drho = T(0), mx = T(0), my = T(0), mz = T(0);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    drho += df[q];
    if (cx(q)) mx += cx(q) > 0 ? df[q] : -df[q];
    if (cy(q)) my += cy(q) > 0 ? df[q] : -df[q];
    if (cz(q)) mz += cz(q) > 0 ? df[q] : -df[q];
  }
  const T rho = PP.rho0 + drho;
  const T inv = T(1) / rho;
  const T ux = (mx + T(0.5) * Fx) * inv, uy = (my + T(0.5) * Fy) * inv, uz = (mz + T(0.5) * Fz) * inv;
  const T usq = ux * ux + uy * uy + uz * uz;
  const T uF = ux * Fx + uy * Fy + uz * Fz;
  const T omega = PP.omega, pref = PP.pref;
  const uint64_t pol_stream = l2_stream(), pol_keep = l2_keep();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const T w = T(wq(q));
    const T cu = T(cx(q)) * ux + T(cy(q)) * uy + T(cz(q)) * uz;
    const T cF = T(cx(q)) * Fx + T(cy(q)) * Fy + T(cz(q)) * Fz;
    const T eq = w * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
    const T src = pref * w * (T(3) * (cF - uF) + T(9) * cu * cF);
    st_hint(fout + (size_t)q * N + i, df[q] - omega * (df[q] - eq) + src, pol_stream);
  }
  st_hint(ub + i, ux, pol_keep);
  st_hint(ub + (size_t)N + i, uy, pol_keep);
  st_hint(ub + (size_t)2 * N + i, uz, pol_keep);
}

template <typename T>
__device__ __forceinline__ void solid_velocity(const DevBox& B, T* __restrict__ ub, int x, int y, int z, int i,
                                               uint8_t m) {
  const DevColloid& C = B.col[(m & IDMASK) - 1];
  T ur[3];
  rigid_velocity_t<T>(B, T(x), T(y), T(z), C.X, C.V, C.W, ur);
#pragma unroll
  for (int a = 0; a < 3; ++a) ub[(size_t)a * B.N + i] = ur[a];
}

// ---------------------------------------------------------------------------
// k_lb: collide/stream with the body force read from memory
// ---------------------------------------------------------------------------
template <typename T, int TY>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 ? 768 : 384) / (TX * TY)) k_lb(
    const DevBox* __restrict__ boxes, const int4* __restrict__ tiles, int ntiles, int zc, int mode,
    double* __restrict__ part) {
  __shared__ DevBox B;
  int cur_box = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = tiles[t];
    load_box(B, boxes, td.x, cur_box);
    if (!B.p.flow_on) continue;
    const PhysT<T>& PP = phys<T>(B);
    const int fpar = B.st->fpar;
    const bool pre = B.st->pre_valid != 0;
    const T* __restrict__ fin = static_cast<const T*>(B.f[fpar]);
    T* __restrict__ fout = static_cast<T*>(B.f[fpar ^ 1]);
    const T* __restrict__ Fb = static_cast<const T*>(B.F);
    T* __restrict__ ub = static_cast<T*>(B.u);
    const int nx = B.nx, ny = B.ny, N = B.N;
    const int x = td.y + threadIdx.x, y = td.z + threadIdx.y;
    const int zend = min(td.w + zc, B.nz);
    if (x >= nx || y >= ny) continue;
    const bool lc = B.p.lc_on != 0;
    for (int z = td.w; z < zend; ++z) {
      const int i = x + nx * (y + ny * z);
      const uint8_t m = B.mask[i];
      if (m & IDMASK) {
        solid_velocity(B, ub, x, y, z, i, m);
        continue;
      }
      T df[NQ];
      pull(B, fin, x, y, z, i, m, pre, df);
      T Fx = PP.g[0], Fy = PP.g[1], Fz = PP.g[2];
      if (lc) {
        Fx += Fb[i];
        Fy += Fb[(size_t)N + i];
        Fz += Fb[(size_t)2 * N + i];
      }
      collide_store(PP, fout, ub, N, i, df, Fx, Fy, Fz);
    }
  }
}

// ---------------------------------------------------------------------------
// x-neighbour values from the adjacent lanes
// ---------------------------------------------------------------------------
// The lanes of a warp hold consecutive x of one row, so the K values of the
// x +- 1 neighbours of a node come from lanes +- 1 by shuffles; a lane whose
// neighbour is not held by the adjacent lane (the tile's edge lanes, the
// periodic wrap, the end of a ragged row) loads it.  All 32 lanes call this.
// xn[0] = x + 1, xn[1] = x - 1 (the order of face_neighbours).
template <typename T, int K, bool CG = false>
__device__ __forceinline__ void x_neighbours(const T* __restrict__ F, size_t N, const T self[K], int lane, int x,
                                             int nx, int row, bool valid, T xn[2][K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    xn[0][k] = __shfl_down_sync(0xffffffffu, self[k], 1);
    xn[1][k] = __shfl_up_sync(0xffffffffu, self[k], 1);
  }
  if (!valid) return;
  if (lane == TX - 1 || x + 1 >= nx) {
    const int j = (x + 1 == nx ? 0 : x + 1) + row;
#pragma unroll
    for (int k = 0; k < K; ++k) xn[0][k] = ldx<CG>(F + (size_t)k * N + j);
  }
  if (lane == 0) {
    const int j = (x == 0 ? nx - 1 : x - 1) + row;
#pragma unroll
    for (int k = 0; k < K; ++k) xn[1][k] = ldx<CG>(F + (size_t)k * N + j);
  }
}

// Values of the thread's own column (x, y) down the z march: at the start of
// a tile, z0 - 1 and z0 (the plane below z0 wraps in a periodic box; beyond a
// wall the value is 0 and unused, such nodes being near nodes).  Each step
// loads z + 1 into pc[3], takes z into pc[0] and z - 1 into pc[4]
// (pc[1], pc[2] are the x-neighbours), and column_roll moves the window up.
template <typename T, int K>
__device__ __forceinline__ void column_start(const DevBox& B, const T* __restrict__ F, int x, int y, int z0,
                                             bool valid, T cz[2][K]) {
  const int zm = z0 > 0 ? z0 - 1 : (B.wall_z ? -1 : B.nz - 1);
  const size_t N = (size_t)B.N;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    cz[0][k] = (valid && zm >= 0) ? ldg(F + (size_t)k * N + x + B.nx * (y + B.ny * zm)) : T(0);
    cz[1][k] = valid ? ldg(F + (size_t)k * N + x + B.nx * (y + B.ny * z0)) : T(0);
  }
}

template <typename T, int K>
__device__ __forceinline__ void column_next(const DevBox& B, const T* __restrict__ F, int x, int y, int z, bool valid,
                                            const T cz[2][K], T pc[5][K]) {
  const int zp = z + 1 < B.nz ? z + 1 : (B.wall_z ? -1 : 0);
  const size_t N = (size_t)B.N;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    pc[0][k] = cz[1][k];
    pc[4][k] = cz[0][k];
    pc[3][k] = (valid && zp >= 0) ? ldg(F + (size_t)k * N + x + B.nx * (y + B.ny * zp)) : T(0);
  }
}

template <typename T, int K>
__device__ __forceinline__ void column_roll(T cz[2][K], const T pc[5][K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    cz[0][k] = pc[0][k];
    cz[1][k] = pc[3][k];
  }
}

// ---------------------------------------------------------------------------
// stored-stress variant: k_stress stores H and P once per fluid node, k_lbp
// takes the body force from the stored P
// ---------------------------------------------------------------------------
// Node i of the stored-stress kernel: gather (surface values at solid or wall
// faces when near), H, P, stores, and for near nodes the colloid LC force.
// A plain node (NEAR_NODE false) takes its own Q and that of its x- and
// z-neighbours from pq (self, x + 1, x - 1, z + 1, z - 1: gathered by the warp
// and rolled down the thread's column) and loads the y-neighbours.
// FP32 node next to a solid or wall: derivatives from the compensated Q
// (near_derivatives_f32), H and P stored, colloid faces summed.  Every node
// of the shell around a colloid or along a wall takes this path: the
// colloid's LC force is a small sum of large face terms, and the body force
// at the boundary links, which sets the hydrodynamic force, is the face
// divergence of the stress of these nodes.  Not inlined, so that the wider
// arithmetic of this rare path does not raise the register count of the
// plain path of the stress kernels.
__device__ __noinline__ void near_stress_f32(const DevBox& B, float* __restrict__ Hb, float* __restrict__ Pb, int x,
                                             int y, int z, int i, int mode, int& my_c, double my_acc[6]) {
  const int N = B.N;
  float qi[5], dq[3][5], lap[5], h[5], p[9], fp;
  near_derivatives_f32(B, x, y, z, i, qi, dq, lap);
  lc_node_d<float, true>(B.pf, qi, dq, lap, h, p, &fp);
#pragma unroll
  for (int c = 0; c < 5; ++c) Hb[(size_t)c * N + i] = h[c];
#pragma unroll
  for (int c = 0; c < 9; ++c) Pb[(size_t)c * N + i] = p[c];
  if (mode & FORCE_ACC) {
    int nb[6], zz[2];
    face_neighbours(B, x, y, z, nb, zz);
    for (int d = 0; d < 6; ++d) {
      const int j = nb[d];
      if (j < 0) continue;
      const uint8_t fj = B.mask[j] & IDMASK;
      if (fj == 0) continue;
      const int ax = d >> 1;
      const float sgn = (d & 1) ? -1.f : 1.f;
      const float pcv[3] = {p[ax], p[3 + ax], p[6 + ax]};
      colloid_face(B, fj - 1, ax, sgn, pcv, x, y, z, my_c, my_acc);
    }
  }
}

template <typename T, bool NEAR_NODE>
__device__ __forceinline__ void stress_node(const DevBox& B, const PhysT<T>& PP, const T* __restrict__ Q,
                                            T* __restrict__ Hb, T* __restrict__ Pb, int x, int y, int z, int i,
                                            uint8_t m, int mode, int& my_c, double my_acc[6],
                                            const T (*pq)[5] = nullptr) {
  if constexpr (NEAR_NODE && sizeof(T) == 4) {
    near_stress_f32(B, Hb, Pb, x, y, z, i, mode, my_c, my_acc);
    return;
  }
  const int N = B.N;
  T qi[5], qn[6][5], h[5], p[9], fp;
  if (NEAR_NODE) {
    gather_q(B, Q, x, y, z, i, m, qi, qn, nullptr);
  } else {
    int nb[6], zz[2];
    face_neighbours(B, x, y, z, nb, zz);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      qi[k] = pq[0][k];
      qn[0][k] = pq[1][k];
      qn[1][k] = pq[2][k];
      qn[4][k] = pq[3][k];
      qn[5][k] = pq[4][k];
    }
#pragma unroll
    for (int d = 2; d < 4; ++d)
#pragma unroll
      for (int k = 0; k < 5; ++k) qn[d][k] = ldg(Q + (size_t)k * N + nb[d]);
  }
  lc_node<T, true>(PP, qi, qn, h, p, &fp);
#pragma unroll
  for (int c = 0; c < 5; ++c) Hb[(size_t)c * N + i] = h[c];
#pragma unroll
  for (int c = 0; c < 9; ++c) Pb[(size_t)c * N + i] = p[c];
  if (NEAR_NODE && (mode & FORCE_ACC)) {
    int nb[6], zz[2];
    face_neighbours(B, x, y, z, nb, zz);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const int j = nb[d];
      if (j < 0) continue;
      const uint8_t fj = B.mask[j] & IDMASK;
      if (fj == 0) continue;
      const int ax = d >> 1;
      const T sgn = (d & 1) ? T(-1) : T(1);
      const T pcv[3] = {p[ax], p[3 + ax], p[6 + ax]};
      colloid_face(B, fj - 1, ax, sgn, pcv, x, y, z, my_c, my_acc);
    }
  }
}

// k_stress: H and P stored once per fluid node.  A warp evaluates its row's
// nodes away from solids and walls together; nodes next to a solid or wall
// (surface values, colloid faces) are queued per warp and evaluated 32 at a
// time, so a row that crosses a colloid does not run the surface path with
// most of its lanes idle.
template <typename T, int TY>
__device__ __forceinline__ void stress_tile(const DevBox& B, const int4 td, int zc, int mode, int (*sq)[2 * TX]) {
  if (!B.p.lc_on) return;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const PhysT<T>& PP = phys<T>(B);
  const T* __restrict__ Q = static_cast<const T*>(B.Q[B.st->qpar]);
  T* __restrict__ Hb = static_cast<T*>(B.H);
  T* __restrict__ Pb = static_cast<T*>(B.P);
  const int nx = B.nx, ny = B.ny;
  const int x = td.y + lane, y = td.z + wy;
  const int zend = min(td.w + zc, B.nz);
  const bool valid = x < nx && y < ny;
  int my_c = -1;
  double my_acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int nq = 0;  // queued near nodes of this warp (warp-uniform)
  T qz[2][5];  // Q of the thread's own column at z - 1 and z, rolled down the z march
  column_start<T, 5>(B, Q, x, y, td.w, valid, qz);
  for (int z = td.w; z < zend; ++z) {
    const int i = x + nx * (y + ny * z);
    const uint8_t m = valid ? B.mask[i] : (uint8_t)1;
    const bool fluid = (m & IDMASK) == 0;
    const bool near = fluid && (m & NEAR);
    T pq[5][5];
    column_next<T, 5>(B, Q, x, y, z, valid, qz, pq);
    x_neighbours<T, 5>(Q, (size_t)B.N, pq[0], lane, x, nx, nx * (y + ny * z), valid, &pq[1]);
    if (fluid && !near) stress_node<T, false>(B, PP, Q, Hb, Pb, x, y, z, i, m, mode, my_c, my_acc, pq);
    const unsigned nb = __ballot_sync(0xffffffffu, near);
    if (nb) {
      if (near) sq[wy][nq + __popc(nb & ((1u << lane) - 1u))] = i;
      nq += __popc(nb);
      __syncwarp();
      if (nq >= TX) {
        const int j = sq[wy][lane];
        const int jx = j % nx, jy = (j / nx) % ny, jz = j / (nx * ny);
        stress_node<T, true>(B, PP, Q, Hb, Pb, jx, jy, jz, j, B.mask[j], mode, my_c, my_acc);
        __syncwarp();
        nq -= TX;
        if (lane < nq) sq[wy][lane] = sq[wy][TX + lane];
        __syncwarp();
      }
    }
    column_roll<T, 5>(qz, pq);
  }
  if (lane < nq) {
    const int j = sq[wy][lane];
    const int jx = j % nx, jy = (j / nx) % ny, jz = j / (nx * ny);
    stress_node<T, true>(B, PP, Q, Hb, Pb, jx, jy, jz, j, B.mask[j], mode, my_c, my_acc);
  }
  __syncwarp();
  if (mode & FORCE_ACC) warp_flush_colloid(B.col, my_c, my_acc, 6);
}

// ---------------------------------------------------------------------------
// two-node paths of the FP32 kernels (boxes of even width)
// ---------------------------------------------------------------------------
// A lane holds the nodes x and x + 1 (x even) of its row, so a warp covers 64
// columns: the fields move as float2, the x-neighbours of the pair come from
// the adjacent lanes by one shuffle per component, and the per-node
// arithmetic of the two nodes runs together in packed FP32x2 (f2).  A pair
// with a node next to a solid or wall sends its fluid nodes through the
// per-warp queue of the one-node path.
__device__ __forceinline__ f2 ld2(const float* p) { return f2(__ldg(reinterpret_cast<const float2*>(p))); }
__device__ __forceinline__ void st2(float* p, f2 v) { *reinterpret_cast<float2*>(p) = v.v; }
__device__ __forceinline__ void st2_keep(float* p, f2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.v.x), "f"(v.v.y), "l"(pol)
               : "memory");
}

template <bool CG>
__device__ __forceinline__ f2 ldx2(const float* p) {
  const float2* q = reinterpret_cast<const float2*>(p);
  if constexpr (CG) return f2(__ldcg(q));
  else return f2(__ldg(q));
}

// The pair's values of a field row shifted by -s (s = +1: the nodes x - 1, x;
// s = -1: x + 1, x + 2), from the float2 v of the nodes x, x + 1 of the same
// row.  All lanes call it; edge lanes load the outside node from src_row.
template <bool CG>
__device__ __forceinline__ f2 shift_pair(f2 v, int s, int lane, bool valid, int x, int nx, const float* src_row) {
  const float left = __shfl_up_sync(0xffffffffu, v.v.y, 1);
  const float right = __shfl_down_sync(0xffffffffu, v.v.x, 1);
  if (s > 0) {
    float l = left;
    if (valid && lane == 0) l = ldx<CG>(src_row + (x == 0 ? nx - 1 : x - 1));
    return f2(l, v.v.x);
  }
  float r = right;
  if (valid && (lane == TX - 1 || x + 2 >= nx)) r = ldx<CG>(src_row + (x + 2 >= nx ? x + 2 - nx : x + 2));
  return f2(v.v.y, r);
}

// Push node j (when cond) onto the warp's queue sq[wy], evaluating 32 queued
// nodes with fn(j) whenever the queue holds 32 or more.  All lanes call it.
template <typename Fn>
__device__ __forceinline__ void queue_push(int (*sq)[2 * TX], int wy, int lane, int& nq, bool cond, int j, Fn fn) {
  const unsigned nb = __ballot_sync(0xffffffffu, cond);
  if (!nb) return;
  if (cond) sq[wy][nq + __popc(nb & ((1u << lane) - 1u))] = j;
  nq += __popc(nb);
  __syncwarp();
  if (nq >= TX) {
    fn(sq[wy][lane]);
    __syncwarp();
    nq -= TX;
    if (lane < nq) sq[wy][lane] = sq[wy][TX + lane];
    __syncwarp();
  }
}

// Stored-stress kernel, two nodes per lane: H and P of the pair from packed
// derivatives (the z-neighbours rolled down the column as in stress_tile).
// The loads of the next plane (mask, the column's z + 1 and the rows y +- 1)
// are issued before the current plane is evaluated, so their latency is
// covered by that plane's arithmetic rather than by other warps.
template <int TY>
__device__ __forceinline__ void stress_tile_pair(const DevBox& B, const int4 td, int zc, int mode,
                                                 int (*sq)[2 * TX]) {
  if (!B.p.lc_on) return;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const float* __restrict__ Q = static_cast<const float*>(B.Q[B.st->qpar]);
  float* __restrict__ Hb = static_cast<float*>(B.H);
  float* __restrict__ Pb = static_cast<float*>(B.P);
  const int nx = B.nx, ny = B.ny, nz = B.nz;
  const size_t N = (size_t)B.N;
  const int x = td.y + 2 * lane, y = td.z + wy;
  const int zend = min(td.w + zc, nz);
  const bool valid = x < nx && y < ny;
  const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
  int my_c = -1;
  double my_acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int nq = 0;
  auto near_fn = [&](int j) {
    stress_node<float, true>(B, B.pf, Q, Hb, Pb, j % nx, (j / nx) % ny, j / (nx * ny), j, B.mask[j], mode, my_c,
                             my_acc);
  };
  f2 qz[2][5];  // the pair's Q at z - 1 and z, rolled down the z march
  f2 pz[5], pyp[5], pym[5];  // next plane's loads: the pair's Q at z + 1, the rows y + 1 and y - 1 at z
  unsigned pm2;              // and the pair's mask bytes at z
  auto fetch = [&](int z) {
    const int zp = z + 1 < nz ? z + 1 : (B.wall_z ? -1 : 0);
    pm2 = valid ? (unsigned)*reinterpret_cast<const uint16_t*>(B.mask + x + nx * (y + ny * z)) : 0x0101u;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      pz[k] = (valid && zp >= 0) ? ld2(Q + k * N + x + nx * (y + ny * zp)) : f2(0.f);
      pyp[k] = valid ? ld2(Q + k * N + x + nx * (yp + ny * z)) : f2(0.f);
      pym[k] = valid ? ld2(Q + k * N + x + nx * (ym + ny * z)) : f2(0.f);
    }
  };
  {
    const int zm = td.w > 0 ? td.w - 1 : (B.wall_z ? -1 : nz - 1);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      qz[0][k] = (valid && zm >= 0) ? ld2(Q + k * N + x + nx * (y + ny * zm)) : f2(0.f);
      qz[1][k] = valid ? ld2(Q + k * N + x + nx * (y + ny * td.w)) : f2(0.f);
    }
  }
  if (td.w < zend) fetch(td.w);
  for (int z = td.w; z < zend; ++z) {
    const int row = nx * (y + ny * z);
    const int i = x + row;
    const unsigned m2 = pm2;
    const uint8_t mA = (uint8_t)(m2 & 0xffu), mB = (uint8_t)(m2 >> 8);
    const bool fA = (mA & IDMASK) == 0, fB = (mB & IDMASK) == 0;
    const bool plain = fA && fB && !(mA & NEAR) && !(mB & NEAR);
    f2 qn[6][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      qn[4][k] = pz[k];
      qn[2][k] = pyp[k];
      qn[3][k] = pym[k];
      qn[5][k] = qz[0][k];
    }
    if (z + 1 < zend) fetch(z + 1);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      qn[0][k] = shift_pair<false>(qz[1][k], -1, lane, valid, x, nx, Q + k * N + row);
      qn[1][k] = shift_pair<false>(qz[1][k], 1, lane, valid, x, nx, Q + k * N + row);
    }
    if (plain) {
      f2 dq[3][5], lap[5], h[5], p[9], fp;
      derivatives(qz[1], qn, dq, lap);
      lc_node_d<f2, true, float>(B.pf, qz[1], dq, lap, h, p, &fp);
      const uint64_t keep = l2_keep();
#pragma unroll
      for (int c = 0; c < 5; ++c) st2_keep(Hb + c * N + i, h[c], keep);
#pragma unroll
      for (int c = 0; c < 9; ++c) st2_keep(Pb + c * N + i, p[c], keep);
    }
    queue_push(sq, wy, lane, nq, fA && !plain, i, near_fn);
    queue_push(sq, wy, lane, nq, fB && !plain, i + 1, near_fn);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      qz[0][k] = qz[1][k];
      qz[1][k] = qn[4][k];
    }
  }
  if (lane < nq) near_fn(sq[wy][lane]);
  __syncwarp();
  if (mode & FORCE_ACC) warp_flush_colloid(B.col, my_c, my_acc, 6);
}

template <typename T, int TY>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 ? 384 : 256) / (TX * TY)) k_stress(
    const DevBox* __restrict__ boxes, const int4* __restrict__ tiles, int ntiles, int zc, int mode,
    double* __restrict__ part) {
  __shared__ DevBox B;
  __shared__ int sq[TY][2 * TX];  // per-warp queue of near fluid nodes
  int cur_box = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = tiles[t];
    load_box(B, boxes, td.x, cur_box);
    if constexpr (sizeof(T) == 4) {
      if (pair_box(B)) {
        stress_tile_pair<TY>(B, td, zc, mode, sq);
        continue;
      }
    }
    stress_tile<T, TY>(B, td, zc, mode, sq);
  }
}

// Body force at fluid node i from the stored stress: the face divergence of
// k_flb, sum over the six faces of +-(face value), the face value the mean of
// the two nodes' P or, across a solid or wall face, P(i).  With six fluid
// neighbours the P(i) halves cancel.
template <typename T, bool CG = false>
__device__ __forceinline__ void stored_force(const DevBox& B, const T* __restrict__ Pb, int x, int y, int z, int i,
                                             uint8_t m, T F[3]) {
  const size_t N = (size_t)B.N;
  int nb[6], zz[2];
  face_neighbours(B, x, y, z, nb, zz);
  if (!(m & NEAR)) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T* Pa = Pb + (size_t)(3 * a) * N;
      F[a] = T(0.5) * ((ldx<CG>(Pa + nb[0]) - ldx<CG>(Pa + nb[1])) + (ldx<CG>(Pa + N + nb[2]) - ldx<CG>(Pa + N + nb[3])) +
                       (ldx<CG>(Pa + 2 * N + nb[4]) - ldx<CG>(Pa + 2 * N + nb[5])));
    }
    return;
  }
  F[0] = F[1] = F[2] = T(0);
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int j = nb[d];
    const bool fluid = j >= 0 && (B.mask[j] & IDMASK) == 0;
    const int ax = d >> 1;
    const T sgn = (d & 1) ? T(-1) : T(1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T* Pc = Pb + (size_t)(3 * a + ax) * N;
      const T pc = ldx<CG>(Pc + i);
      const T face = fluid ? T(0.5) * (pc + ldx<CG>(Pc + j)) : pc;
      F[a] += sgn * face;
    }
  }
}

// One fluid node of k_lbp: pull (bounce-back only for near nodes), body force
// from the stored P, collide, store.  For a plain node the mask handed down
// has the near bit cleared, which removes the neighbour checks at compile time.
template <typename T, bool NEAR_NODE, bool CG = false>
__device__ __forceinline__ void lbp_node(const DevBox& B, const PhysT<T>& PP, const T* __restrict__ fin,
                                         T* __restrict__ fout, const T* __restrict__ Pb, T* __restrict__ ub, int x,
                                         int y, int z, int i, uint8_t m, bool pre, bool lc) {
  const uint8_t mm = NEAR_NODE ? m : (uint8_t)(m & (uint8_t)~NEAR);
  T df[NQ];
  pull(B, fin, x, y, z, i, mm, pre, df);
  T Fx = PP.g[0], Fy = PP.g[1], Fz = PP.g[2];
  if (lc) {
    T Fv[3];
    stored_force<T, CG>(B, Pb, x, y, z, i, mm, Fv);
    Fx += Fv[0];
    Fy += Fv[1];
    Fz += Fv[2];
  }
  collide_store(PP, fout, ub, B.N, i, df, Fx, Fy, Fz);
}

// k_lbp: like k_stress, a warp collides the plain fluid nodes of its row
// together and queues the nodes next to a solid or wall (bounce-back links,
// solid faces of the force) in shared memory, 32 at a time.
template <typename T, int TY, bool CG>
__device__ __forceinline__ void lbp_tile(const DevBox& B, const int4 td, int zc, int (*sq)[2 * TX]) {
  if (!B.p.flow_on) return;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const PhysT<T>& PP = phys<T>(B);
  const int fpar = B.st->fpar;
  const bool pre = B.st->pre_valid != 0;
  const T* __restrict__ fin = static_cast<const T*>(B.f[fpar]);
  T* __restrict__ fout = static_cast<T*>(B.f[fpar ^ 1]);
  const T* __restrict__ Pb = static_cast<const T*>(B.P);
  T* __restrict__ ub = static_cast<T*>(B.u);
  const int nx = B.nx, ny = B.ny;
  const int x = td.y + lane, y = td.z + wy;
  const int zend = min(td.w + zc, B.nz);
  const bool valid = x < nx && y < ny;
  const bool lc = B.p.lc_on != 0;
  int nq = 0;
  for (int z = td.w; z < zend; ++z) {
    const int i = x + nx * (y + ny * z);
    const uint8_t m = valid ? B.mask[i] : (uint8_t)0;
    const bool fluid = valid && (m & IDMASK) == 0;
    const bool near = fluid && (m & NEAR);
    if (valid && !fluid) solid_velocity(B, ub, x, y, z, i, m);
    if (fluid && !near) lbp_node<T, false, CG>(B, PP, fin, fout, Pb, ub, x, y, z, i, m, pre, lc);
    const unsigned nb = __ballot_sync(0xffffffffu, near);
    if (nb) {
      if (near) sq[wy][nq + __popc(nb & ((1u << lane) - 1u))] = i;
      nq += __popc(nb);
      __syncwarp();
      if (nq >= TX) {
        const int j = sq[wy][lane];
        lbp_node<T, true, CG>(B, PP, fin, fout, Pb, ub, j % nx, (j / nx) % ny, j / (nx * ny), j, B.mask[j], pre, lc);
        __syncwarp();
        nq -= TX;
        if (lane < nq) sq[wy][lane] = sq[wy][TX + lane];
        __syncwarp();
      }
    }
  }
  if (lane < nq) {
    const int j = sq[wy][lane];
    lbp_node<T, true, CG>(B, PP, fin, fout, Pb, ub, j % nx, (j / nx) % ny, j / (nx * ny), j, B.mask[j], pre, lc);
  }
  __syncwarp();
}

template <typename T, int TY>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 ? 768 : 384) / (TX * TY)) k_lbp(
    const DevBox* __restrict__ boxes, const int4* __restrict__ tiles, int ntiles, int zc, int mode,
    double* __restrict__ part) {
  __shared__ DevBox B;
  __shared__ int sq[TY][2 * TX];
  int cur_box = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = tiles[t];
    load_box(B, boxes, td.x, cur_box);
    lbp_tile<T, TY, false>(B, td, zc, sq);
  }
}

// ---------------------------------------------------------------------------
// k_flb: stress + body force + collide/stream fused (the step kernel)
// ---------------------------------------------------------------------------
// Tile: 32 x BY interior columns marching z.  Threads: 32*(BY+2) cover the
// stress positions of the tile rows and the two y-halo rows (whole warps),
// one more warp the two x-halo columns, so every halo position of a plane is
// computed in a single pass.  Warps 1..BY then run the body force and the LB
// collide of their interior node; the stress never leaves shared memory and
// the body force never reaches HBM.
template <typename T, int BY>
__global__ void __launch_bounds__(32 * (BY + 3), (sizeof(T) == 4 && BY <= 4) ? 2 : 1) k_flb(
    const DevBox* __restrict__ boxes, const int4* __restrict__ tiles, int ntiles, int zc, int mode,
    double* __restrict__ part) {
  constexpr int HX = TX + 2, HY = BY + 2, HP = HX * HY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sP = reinterpret_cast<T*>(smem_raw);
  uint8_t* sFl = smem_raw + sizeof(T) * 27 * HP;
  __shared__ DevBox B;
  const int tid = threadIdx.x;
  // this thread's stress position (hx, hy) in the halo'd plane, or none
  int hx, hy;
  if (tid < 32 * HY) {
    hx = 1 + (tid & 31);
    hy = tid >> 5;
  } else {
    const int k = tid - 32 * HY;
    hx = k < HY ? 0 : (k < 2 * HY ? HX - 1 : -1);
    hy = k < HY ? k : k - HY;
  }
  const int pidx = hx >= 0 ? hx + HX * hy : -1;
  const bool lbthread = tid >= 32 && tid < 32 * (BY + 1);
  const int tx = tid & 31, ty = (tid >> 5) - 1;

  int cur_box = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = tiles[t];
    load_box(B, boxes, td.x, cur_box);
    const PhysT<T>& PP = phys<T>(B);
    const bool lc = B.p.lc_on != 0, flow = B.p.flow_on != 0;
    if (!flow && !lc) continue;
    int my_c = -1;
    double my_acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const T* __restrict__ Q = static_cast<const T*>(B.Q[B.st->qpar]);
    const int fpar = B.st->fpar;
    const bool pre = B.st->pre_valid != 0;
    const T* __restrict__ fin = static_cast<const T*>(B.f[fpar]);
    T* __restrict__ fout = static_cast<T*>(B.f[fpar ^ 1]);
    T* __restrict__ ub = static_cast<T*>(B.u);
    const int x0 = td.y, y0 = td.z, z0 = td.w;
    const int nx = B.nx, ny = B.ny, nz = B.nz, N = B.N;
    const int vx = min(TX, nx - x0), vy = min(BY, ny - y0);
    const int zend = min(z0 + zc, nz);
    const bool mypos = pidx >= 0 && hx <= vx + 1 && hy <= vy + 1;
    const int gx = wrapn(x0 - 1 + hx, nx), gy = wrapn(y0 - 1 + hy, ny);
    const bool myint = lbthread && tx < vx && ty < vy;
    for (int k = z0 - 1; k <= zend; ++k) {
      const int slot = (k - z0 + 1) % 3;
      if (lc && mypos) {
        const bool wallplane = B.wall_z && (k < 0 || k >= nz);
        const int kk = B.wall_z ? k : wrapn(k, nz);
        double dummy = 0.0;
        const bool inner = hx >= 1 && hx <= vx && hy >= 1 && hy <= vy && k >= z0 && k < zend;
        sFl[slot * HP + pidx] =
            wallplane ? WALLFLAG
                      : stress_at(B, PP, Q, gx, gy, kk, sP + slot * 9 * HP + pidx, HP, false, &dummy,
                                  inner ? static_cast<T*>(B.H) : (T*)nullptr);
      }
      __syncthreads();
      if (k >= z0 + 1 && myint) {
        const int kc = k - 1;
        const int x = x0 + tx, y = y0 + ty;
        const int i = x + nx * (y + ny * kc);
        const uint8_t m = B.mask[i];
        if (m & IDMASK) {
          if (flow) solid_velocity(B, ub, x, y, kc, i, m);
        } else {
          T Fv[3] = {T(0), T(0), T(0)};
          if (lc)
            face_force(B, sP, sFl, HP, HX, (k - z0) % 3, (k - z0 - 1) % 3, slot, (tx + 1) + HX * (ty + 1), x, y, kc,
                       (mode & FORCE_ACC) != 0, Fv, my_c, my_acc);
          if (flow) {
            T df[NQ];
            pull(B, fin, x, y, kc, i, m, pre, df);
            collide_store(PP, fout, ub, N, i, df, Fv[0] + PP.g[0], Fv[1] + PP.g[1], Fv[2] + PP.g[2]);
          }
        }
      }
      __syncthreads();
    }
    if (mode & FORCE_ACC) warp_flush_colloid(B.col, my_c, my_acc, 6);
  }
}

// ---------------------------------------------------------------------------
// k_lc: Beris-Edwards update
// ---------------------------------------------------------------------------
// Beris-Edwards update of fluid node i (Eq. 2): co-rotation from the central
// velocity gradient, upwind advective fluxes through the faces (zero across
// solid or wall faces, which only near nodes have), H stored by the stress
// kernel of this step; Q^{n+1} stored, residual folded into (rsum, rmax).
// A plain node (NEAR_NODE false) takes its own Q and u and those of its
// x-neighbours from pq and pu (self, x + 1, x - 1; gathered by the warp).
// Holding the z-neighbours in registers down the z march, as the stress
// kernel does, pushed this kernel past its 96-register cap (spills, 76 us
// against 71 us).
template <typename T, bool NEAR_NODE, bool CG = false>
__device__ __forceinline__ void lc_update_node(const DevBox& B, const PhysT<T>& PP, const T* __restrict__ Q,
                                               T* __restrict__ Qo, const __nv_bfloat16* __restrict__ Lin,
                                               __nv_bfloat16* __restrict__ Lout, const T* __restrict__ U, int x,
                                               int y, int z, int i, uint8_t m, T& rsum, T& rmax,
                                               const T (*pq)[5] = nullptr, const T (*pu)[3] = nullptr,
                                               const float* plo = nullptr) {
  const int N = B.N;
  // BF16 remainder of the node's own Q (FP32 storage), loaded with the other
  // inputs so that its latency overlaps theirs
  float lo[5];
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int c = 0; c < 5; ++c) lo[c] = NEAR_NODE ? __bfloat162float(Lin[(size_t)c * N + i]) : plo[c];
  }
  const T Gam = PP.Gamma, xi = PP.xi;
  // H of this node was stored by the stress kernel of this step; Q of the
  // fluid face neighbours is needed only for the advective fluxes (zero
  // across solid faces), so no surface values are formed here
  const T* __restrict__ Hb = static_cast<const T*>(B.H);
  T qi[5], qn[6][5], h[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    qi[c] = NEAR_NODE ? ldg(Q + (size_t)c * N + i) : pq[0][c];
    h[c] = ldx<CG>(Hb + (size_t)c * N + i);
  }
  int nb[6], zz[2];
  face_neighbours(B, x, y, z, nb, zz);
  T ui[3], un[6][3];
  bool fl[6];
#pragma unroll
  for (int a = 0; a < 3; ++a) ui[a] = NEAR_NODE ? ldx<CG>(U + (size_t)a * N + i) : pu[0][a];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int j = nb[d];
    fl[d] = !NEAR_NODE || (j >= 0 && (B.mask[j] & IDMASK) == 0);
    if (!NEAR_NODE && d < 2) {
#pragma unroll
      for (int a = 0; a < 3; ++a) un[d][a] = pu[1 + d][a];
#pragma unroll
      for (int c = 0; c < 5; ++c) qn[d][c] = pq[1 + d][c];
      continue;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) un[d][a] = (!NEAR_NODE || j >= 0) ? ldx<CG>(U + (size_t)a * N + j) : T(0);
#pragma unroll
    for (int c = 0; c < 5; ++c) qn[d][c] = fl[d] ? ldg(Q + (size_t)c * N + j) : T(0);
  }
  // velocity gradient W_ab = d_b u_a
  T W[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) W[a][b] = T(0.5) * (un[2 * b][a] - un[2 * b + 1][a]);
  // advective fluxes through the six faces (zero across solid faces)
  T adv[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    if (!fl[d]) continue;
    const int ax = d >> 1;
    const T uf = T(0.5) * (ui[ax] + un[d][ax]);
    const bool plus = (d & 1) == 0;
    // + face: upwind is i when uf > 0; - face: upwind is the neighbour when uf > 0
    const bool take_i = plus ? (uf > T(0)) : !(uf > T(0));
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const T fl_ = uf * (take_i ? qi[k] : qn[d][k]);
      adv[k] += plus ? fl_ : -fl_;
    }
  }
  // co-rotation S = xi (D Qt + Qt D) + (Om Q - Q Om) - 2 xi Qt Tr(Q W), Qt = Q + I/3
  T D[3][3], Om[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      D[a][b] = T(0.5) * (W[a][b] + W[b][a]);
      Om[a][b] = T(0.5) * (W[a][b] - W[b][a]);
    }
  T trQW = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) trQW += qab(qi, a, b) * D[a][b];
  T dQ[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c)
        s += xi * (D[a][c] * qab(qi, c, b) + qab(qi, a, c) * D[c][b]) + Om[a][c] * qab(qi, c, b) -
             qab(qi, a, c) * Om[c][b];
      s += xi * T(2) / T(3) * D[a][b];
      s -= T(2) * xi * (qab(qi, a, b) + (a == b ? T(1) / T(3) : T(0))) * trQW;
      dQ[a][b] = s;
    }
  const T tr = dQ[0][0] + dQ[1][1] + dQ[2][2];
  const int ia[5] = {0, 0, 0, 1, 1}, ib[5] = {0, 1, 2, 1, 2};
  if constexpr (sizeof(T) == 4) {
    // H was evaluated at hi; the stored Q is hi + lo.  Add the local part of
    // H(hi + lo) - H(hi) to first order: the bulk terms' derivative at hi
    // applied to lo, and lo's own term -6 K lo of the Laplacian (the
    // neighbours' lo enter K lap and the gradient terms at the ~1e-9 level).
    // Without it the relaxation stalls where A0 lo ~ the residual.
    const T A0 = PP.A0, g = PP.gamma, K = PP.K, q0 = PP.q0;
    T Qm[3][3], Lm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        Qm[a][b] = qab(qi, a, b);
        Lm[a][b] = qab(lo, a, b);
      }
    T trq2 = T(0), trql = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        trq2 += Qm[a][b] * Qm[a][b];
        trql += Qm[a][b] * Lm[a][b];
      }
    const T cb = -A0 * (T(1) - g / T(3)) - A0 * g * trq2 - T(4) * K * q0 * q0 - T(6) * K;
    const T A0g = A0 * g;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int a = ia[k], b = ib[k];
      T ql = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) ql += Qm[a][c] * Lm[c][b] + Lm[a][c] * Qm[c][b];
      if (a == b) ql -= T(2) / T(3) * trql;
      h[k] += cb * lo[k] + A0g * ql - T(2) * A0g * trql * qi[k];
    }
  }
  T d5[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    T v = Gam * h[k] + dQ[ia[k]][ib[k]] - adv[k];
    if (ia[k] == ib[k]) v -= tr / T(3);
    d5[k] = v;
    if constexpr (sizeof(T) == 4) {
      // compensated FP32 storage: hi + lo + increment carried exactly into hi, to BF16 in lo
      float hi;
      __nv_bfloat16 lo_out;
      add_compensated(qi[k], lo[k], v, hi, lo_out);
      Qo[(size_t)k * N + i] = hi;
      Lout[(size_t)k * N + i] = lo_out;
    } else {
      Qo[(size_t)k * N + i] = qi[k] + v;
    }
  }
  const T dzz = -d5[0] - d5[3];
  rsum += d5[0] * d5[0] + d5[3] * d5[3] + dzz * dzz + T(2) * (d5[1] * d5[1] + d5[2] * d5[2] + d5[4] * d5[4]);
  T mx = fabs(dzz);
#pragma unroll
  for (int k = 0; k < 5; ++k) mx = fmax(mx, fabs(d5[k]));
  rmax = fmax(rmax, mx);
}

// k_lc: Beris-Edwards update; plain nodes of a warp's row together, nodes
// next to a solid or wall queued and updated 32 at a time.  part (if non-null)
// receives the tile's residual partials (sum of squares, max), one record per
// warp (TY records per tile).
template <typename T, int TY, bool CG>
__device__ __forceinline__ void lc_tile(const DevBox& B, const int4 td, int zc, double* part, int (*sq)[2 * TX]) {
  if (!B.p.lc_on) return;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int qpar = B.st->qpar;
  const T* __restrict__ Q = static_cast<const T*>(B.Q[qpar]);
  T* __restrict__ Qo = static_cast<T*>(B.Q[qpar ^ 1]);
  const __nv_bfloat16* __restrict__ Lin = B.Qlo[qpar];
  __nv_bfloat16* __restrict__ Lout = B.Qlo[qpar ^ 1];
  const T* __restrict__ U = static_cast<const T*>(B.u);
  const int nx = B.nx, ny = B.ny;
  const int x = td.y + lane, y = td.z + wy;
  const int zend = min(td.w + zc, B.nz);
  const bool valid = x < nx && y < ny;
  const PhysT<T>& PP = phys<T>(B);
  T rsum = T(0), rmax = T(0);  // per-thread residual (sum of squares, max), in T
  int nq = 0;
  for (int z = td.w; z < zend; ++z) {
    const int i = x + nx * (y + ny * z);
    const uint8_t m = valid ? B.mask[i] : (uint8_t)1;
    const bool fluid = (m & IDMASK) == 0;
    const bool near = fluid && (m & NEAR);
    T pq[3][5], pu[3][3];
    float plo[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) pq[0][k] = valid ? ldg(Q + (size_t)k * B.N + i) : T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) pu[0][a] = valid ? ldx<CG>(U + (size_t)a * B.N + i) : T(0);
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int k = 0; k < 5; ++k) plo[k] = (valid && fluid && !near) ? __bfloat162float(Lin[(size_t)k * B.N + i]) : 0.f;
    }
    const int row = nx * (y + ny * z);
    x_neighbours<T, 5>(Q, (size_t)B.N, pq[0], lane, x, nx, row, valid, &pq[1]);
    x_neighbours<T, 3, CG>(U, (size_t)B.N, pu[0], lane, x, nx, row, valid, &pu[1]);
    if (fluid && !near)
      lc_update_node<T, false, CG>(B, PP, Q, Qo, Lin, Lout, U, x, y, z, i, m, rsum, rmax, pq, pu, plo);
    const unsigned nb = __ballot_sync(0xffffffffu, near);
    if (nb) {
      if (near) sq[wy][nq + __popc(nb & ((1u << lane) - 1u))] = i;
      nq += __popc(nb);
      __syncwarp();
      if (nq >= TX) {
        const int j = sq[wy][lane];
        lc_update_node<T, true, CG>(B, PP, Q, Qo, Lin, Lout, U, j % nx, (j / nx) % ny, j / (nx * ny), j, B.mask[j],
                                    rsum, rmax);
        __syncwarp();
        nq -= TX;
        if (lane < nq) sq[wy][lane] = sq[wy][TX + lane];
        __syncwarp();
      }
    }
  }
  if (lane < nq) {
    const int j = sq[wy][lane];
    lc_update_node<T, true, CG>(B, PP, Q, Qo, Lin, Lout, U, j % nx, (j / nx) % ny, j / (nx * ny), j, B.mask[j], rsum,
                                rmax);
  }
  __syncwarp();
  if (part) warp_residual<T>(part, wy, lane, rsum, rmax);
}

// Q update, two nodes per lane (FP32 boxes of even width; tiles 64 wide): the
// Beris-Edwards update of lc_update_node for the nodes x, x + 1 at once, in
// packed FP32x2 arithmetic, with Q, u, H and the BF16 remainder of Q moved as
// pairs.  The upwind choice of each face flux is taken per node.
__device__ __forceinline__ f2 sel2(bool ca, bool cb, f2 a, f2 b) {
  return f2(ca ? a.v.x : b.v.x, cb ? a.v.y : b.v.y);
}

__device__ __forceinline__ void lc_update_pair(const DevBox& B, float* __restrict__ Qo,
                                               __nv_bfloat16* __restrict__ Lout, int i, const f2 qi[5],
                                               const f2 qn[6][5], const f2 ui[3], const f2 un[6][3], const f2 h_[5],
                                               const f2 lo[5], float& rsum, float& rmax) {
  const PhysT<float>& PP = B.pf;
  const size_t N = (size_t)B.N;
  const float Gam = PP.Gamma, xi = PP.xi;
  f2 h[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) h[k] = h_[k];
  // velocity gradient W_ab = d_b u_a
  f2 W[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) W[a][b] = f2(0.5f * (un[2 * b][a] - un[2 * b + 1][a]));
  // upwind advective fluxes through the six faces (no solid faces here)
  f2 adv[5] = {f2(0.f), f2(0.f), f2(0.f), f2(0.f), f2(0.f)};
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int ax = d >> 1;
    const f2 uf = f2(0.5f * (ui[ax] + un[d][ax]));
    const bool plus = (d & 1) == 0;
    const bool pa = uf.v.x > 0.f, pb = uf.v.y > 0.f;
    const bool ta = plus ? pa : !pa, tb = plus ? pb : !pb;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const f2 up = sel2(ta, tb, qi[k], qn[d][k]);
      adv[k] = plus ? adv[k] + uf * up : adv[k] - uf * up;
    }
  }
  // co-rotation S = xi (D Qt + Qt D) + (Om Q - Q Om) - 2 xi Qt Tr(Q W), Qt = Q + I/3
  f2 D[3][3], Om[3][3], Qm[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      D[a][b] = f2(0.5f * (W[a][b] + W[b][a]));
      Om[a][b] = f2(0.5f * (W[a][b] - W[b][a]));
      Qm[a][b] = qab(qi, a, b);
    }
  f2 trQW = f2(0.f);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) trQW = trQW + Qm[a][b] * D[a][b];
  const int ia[5] = {0, 0, 0, 1, 1}, ib[5] = {0, 1, 2, 1, 2};
  const float twoxi = 2.f * xi, xi23 = 2.f * xi / 3.f, third = 1.f / 3.f;
  f2 dQ[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      f2 sacc = f2(0.f);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const f2 dq = D[a][c] * Qm[c][b] + Qm[a][c] * D[c][b];
        sacc = sacc + xi * dq;
        sacc = sacc + Om[a][c] * Qm[c][b];
        sacc = sacc - Qm[a][c] * Om[c][b];
      }
      sacc = sacc + xi23 * D[a][b];
      const f2 qt = a == b ? Qm[a][b] + third : Qm[a][b];
      sacc = sacc - twoxi * (qt * trQW);
      dQ[a][b] = sacc;
    }
  const f2 tr = dQ[0][0] + dQ[1][1] + dQ[2][2];
  {
    // local part of H(hi + lo) - H(hi) to first order (as lc_update_node)
    const float A0 = PP.A0, g = PP.gamma, K = PP.K, q0 = PP.q0;
    f2 Lm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Lm[a][b] = qab(lo, a, b);
    f2 trq2 = f2(0.f), trql = f2(0.f);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        trq2 = trq2 + Qm[a][b] * Qm[a][b];
        trql = trql + Qm[a][b] * Lm[a][b];
      }
    const float A0g = A0 * g;
    const f2 cb = (-A0 * (1.f - g / 3.f) - 4.f * K * q0 * q0 - 6.f * K) - A0g * trq2;
    const f2 trql2 = f2(2.f * A0g * trql);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int a = ia[k], b = ib[k];
      f2 ql = f2(0.f);
#pragma unroll
      for (int c = 0; c < 3; ++c) ql = ql + Qm[a][c] * Lm[c][b] + Lm[a][c] * Qm[c][b];
      if (a == b) ql = ql - (2.f / 3.f) * trql;
      h[k] = h[k] + cb * lo[k] + A0g * ql - trql2 * qi[k];
    }
  }
  f2 d5[5];
  const f2 tr3 = f2(third * tr);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    f2 v = Gam * h[k] + dQ[ia[k]][ib[k]] - adv[k];
    if (ia[k] == ib[k]) v = v - tr3;
    d5[k] = v;
    // compensated storage: hi + lo + v carried exactly into (hi, lo) (two-sum)
    const f2 sv = lo[k] + v;
    const f2 hn = qi[k] + sv;
    const f2 bb = hn - qi[k];
    const f2 err = (qi[k] - (hn - bb)) + (sv - bb);
    st2(Qo + (size_t)k * N + i, hn);
    *reinterpret_cast<__nv_bfloat162*>(Lout + (size_t)k * N + i) = __float22bfloat162_rn(err.v);
  }
  const f2 dzz = -(d5[0] + d5[3]);
  const f2 r2 = d5[0] * d5[0] + d5[3] * d5[3] + dzz * dzz + 2.f * (d5[1] * d5[1] + d5[2] * d5[2] + d5[4] * d5[4]);
  rsum += r2.v.x + r2.v.y;
  float mx = fmaxf(fabsf(dzz.v.x), fabsf(dzz.v.y));
#pragma unroll
  for (int k = 0; k < 5; ++k) mx = fmaxf(mx, fmaxf(fabsf(d5[k].v.x), fabsf(d5[k].v.y)));
  rmax = fmaxf(rmax, mx);
}

template <int TY, bool CG>
__device__ __forceinline__ void lc_tile_pair(const DevBox& B, const int4 td, int zc, double* part,
                                             int (*sq)[2 * TX]) {
  if (!B.p.lc_on) return;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int qpar = B.st->qpar;
  const float* __restrict__ Q = static_cast<const float*>(B.Q[qpar]);
  float* __restrict__ Qo = static_cast<float*>(B.Q[qpar ^ 1]);
  const __nv_bfloat16* __restrict__ Lin = B.Qlo[qpar];
  __nv_bfloat16* __restrict__ Lout = B.Qlo[qpar ^ 1];
  const float* __restrict__ U = static_cast<const float*>(B.u);
  const float* __restrict__ Hb = static_cast<const float*>(B.H);
  const int nx = B.nx, ny = B.ny, nz = B.nz;
  const size_t N = (size_t)B.N;
  const int x = td.y + 2 * lane, y = td.z + wy;
  const int zend = min(td.w + zc, nz);
  const bool valid = x < nx && y < ny;
  const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
  float rsum = 0.f, rmax = 0.f;
  int nq = 0;
  auto near_fn = [&](int j) {
    lc_update_node<float, true, CG>(B, B.pf, Q, Qo, Lin, Lout, U, j % nx, (j / nx) % ny, j / (nx * ny), j, B.mask[j],
                                    rsum, rmax);
  };
  for (int z = td.w; z < zend; ++z) {
    const int row = nx * (y + ny * z);
    const int i = x + row;
    const unsigned m2 = valid ? (unsigned)*reinterpret_cast<const uint16_t*>(B.mask + i) : 0x0101u;
    const uint8_t mA = (uint8_t)(m2 & 0xffu), mB = (uint8_t)(m2 >> 8);
    const bool fA = (mA & IDMASK) == 0, fB = (mB & IDMASK) == 0;
    const bool plain = fA && fB && !(mA & NEAR) && !(mB & NEAR);
    f2 qi[5], ui[3], qn[6][5], un[6][3];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      qi[k] = valid ? ldx2<false>(Q + k * N + i) : f2(0.f);
      qn[0][k] = shift_pair<false>(qi[k], -1, lane, valid, x, nx, Q + k * N + row);
      qn[1][k] = shift_pair<false>(qi[k], 1, lane, valid, x, nx, Q + k * N + row);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ui[a] = valid ? ldx2<CG>(U + a * N + i) : f2(0.f);
      un[0][a] = shift_pair<CG>(ui[a], -1, lane, valid, x, nx, U + a * N + row);
      un[1][a] = shift_pair<CG>(ui[a], 1, lane, valid, x, nx, U + a * N + row);
    }
    if (plain) {
      const int zp = z + 1 == nz ? 0 : z + 1, zm = z == 0 ? nz - 1 : z - 1;  // no wall next to a plain node
      const int jr[4] = {x + nx * (yp + ny * z), x + nx * (ym + ny * z), x + nx * (y + ny * zp),
                         x + nx * (y + ny * zm)};
      f2 h[5], lo[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
#pragma unroll
        for (int d = 0; d < 4; ++d) qn[2 + d][k] = ldx2<false>(Q + k * N + jr[d]);
        h[k] = ldx2<CG>(Hb + k * N + i);
        lo[k] = f2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(Lin + k * N + i)));
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 4; ++d) un[2 + d][a] = ldx2<CG>(U + a * N + jr[d]);
      lc_update_pair(B, Qo, Lout, i, qi, qn, ui, un, h, lo, rsum, rmax);
    }
    queue_push(sq, wy, lane, nq, valid && fA && !plain, i, near_fn);
    queue_push(sq, wy, lane, nq, valid && fB && !plain, i + 1, near_fn);
  }
  if (lane < nq) near_fn(sq[wy][lane]);
  __syncwarp();
  if (part) warp_residual<float>(part, wy, lane, rsum, rmax);
}

template <typename T, int TY>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 ? 512 : 256) / (TX * TY)) k_lc(
    const DevBox* __restrict__ boxes, const int4* __restrict__ tiles, int ntiles, int zc, int mode,
    double* __restrict__ part) {
  __shared__ DevBox B;
  __shared__ int sq[TY][2 * TX];
  int cur_box = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = tiles[t];
    load_box(B, boxes, td.x, cur_box);
    double* pt = (mode & LC_RESID) ? part + 2 * (size_t)t * TY : nullptr;
    if constexpr (sizeof(T) == 4) {
      if (pair_box(B)) {
        lc_tile_pair<TY, false>(B, td, zc, pt, sq);
        continue;
      }
    }
    lc_tile<T, TY, false>(B, td, zc, pt, sq);
  }
}

// ---------------------------------------------------------------------------
// k_links: momentum exchange on the boundary links
// ---------------------------------------------------------------------------
// Per link (fluid r, direction b into colloid c): dp = c_b (2 df*_b(r) -
// 6 w_b rho0 c_b.u_b), u_b the rigid velocity at r + c_b/2; torque
// (r + c_b/2 - X) x dp.  The constant w_b rho0 part of 2 f*_b sums to zero
// over a closed surface and is left out.
// One chunk of links (box record B, first link l0, count n) by all threads of
// the block; sblk holds 18 doubles, sc0 one int of shared memory.
template <typename T, bool CG>
__device__ __forceinline__ void links_chunk(const DevBox& B, int l0, int n, double* sblk, int* sc0) {
  if (!B.p.flow_on) return;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const int nl = *B.nlinks;
  for (int base = l0; base < l0 + n; base += nthr) {
    const int l = base + tid;
    int my_c = -1;
    bool mob = false;
    // dp (3), torque (3), then for mobile colloids the drag tensors zv, zw (6 + 6)
    double v[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) v[k] = 0.0;
    // the sub-chunk's first colloid is summed in shared memory (links are sorted by colloid)
    __syncthreads();
    if (tid < 18) sblk[tid] = 0.0;
    if (tid == 0) *sc0 = (base < nl && base < B.nlinks_cap) ? (int)B.link_col[base] : -1;
    __syncthreads();
    if (l < l0 + n && l < nl && l < B.nlinks_cap) {
      const int i = B.link_node[l];
      const int q = B.link_dir[l];
      const int c = B.link_col[l];
      const T* fout = static_cast<const T*>(B.f[B.st->fpar ^ 1]);
      const double dfq = (double)ldx<CG>(fout + (size_t)q * B.N + i);
      const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
      int qx = 0, qy = 0, qz = 0;
      switch (q) {
#define LCLB_CASE(k) case k: qx = cx(k); qy = cy(k); qz = cz(k); break;
        LCLB_CASE(1) LCLB_CASE(2) LCLB_CASE(3) LCLB_CASE(4) LCLB_CASE(5) LCLB_CASE(6) LCLB_CASE(7) LCLB_CASE(8)
        LCLB_CASE(9) LCLB_CASE(10) LCLB_CASE(11) LCLB_CASE(12) LCLB_CASE(13) LCLB_CASE(14) LCLB_CASE(15)
        LCLB_CASE(16) LCLB_CASE(17) LCLB_CASE(18)
#undef LCLB_CASE
        default: break;
      }
      const double w = (q <= 6) ? 1.0 / 18.0 : 1.0 / 36.0;
      const DevColloid& C = B.col[c];
      double d[3], ubv[3];
      disp(B, x + 0.5 * qx, y + 0.5 * qy, z + 0.5 * qz, C.X, d);
      rigid_velocity(C.V, C.W, d, ubv);
      const double corr = 6.0 * w * B.p.rho0 * (qx * ubv[0] + qy * ubv[1] + qz * ubv[2]);
      const double mag = 2.0 * dfq - corr;
      const double dp[3] = {qx * mag, qy * mag, qz * mag};
      const double tq[3] = {d[1] * dp[2] - d[2] * dp[1], d[2] * dp[0] - d[0] * dp[2], d[0] * dp[1] - d[1] * dp[0]};
      my_c = c;
      for (int a = 0; a < 3; ++a) {
        v[a] = dp[a];
        v[3 + a] = tq[a];
      }
      mob = C.mobile != 0;
      if (mob) {
        // the part of dp linear in the rigid velocity, -6 w rho0 c (c.(V + W x d)):
        // coefficients 6 w rho0 c c (V-V) and 6 w rho0 (d x c)(d x c) (W-W)
        const double zk = 6.0 * w * B.p.rho0;
        const double cc[3] = {(double)qx, (double)qy, (double)qz};
        const double rc[3] = {d[1] * cc[2] - d[2] * cc[1], d[2] * cc[0] - d[0] * cc[2], d[0] * cc[1] - d[1] * cc[0]};
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          v[6 + k] = zk * cc[ia[k]] * cc[ib[k]];
          v[12 + k] = zk * rc[ia[k]] * rc[ib[k]];
        }
      }
    }
    const int c0 = *sc0;
    const bool main = (my_c == c0) && c0 >= 0;
    const bool warp_main = __all_sync(0xffffffffu, main || my_c < 0);
    const bool warp_mob = __any_sync(0xffffffffu, mob);
    if (warp_main) {
#pragma unroll
      for (int k = 0; k < 18; ++k) {
        if (k >= 6 && !warp_mob) break;
        const double t = warp_sum(v[k]);
        if ((tid & 31) == 0 && t != 0.0) atomicAdd(&sblk[k], t);
      }
    } else {
      warp_flush_colloid<6>(B.col, my_c, v, 0);
      if (warp_mob) warp_flush_colloid<12>(B.col, mob ? my_c : -1, v + 6, 12);
    }
    __syncthreads();
    if (tid < 18 && c0 >= 0 && sblk[tid] != 0.0) atomicAdd(&B.col[c0].acc[tid < 6 ? tid : tid + 6], sblk[tid]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_links(const DevBox* __restrict__ boxes, const int2* __restrict__ chunks,
                                               int nchunks) {
  __shared__ DevBox B;
  __shared__ double sblk[18];
  __shared__ int sc0;
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int2 cd = chunks[ch];
    load_box(B, boxes, cd.x);
    links_chunk<T, false>(B, cd.y, LINK_CHUNK, sblk, &sc0);
  }
}

// x = A^{-1} b for a symmetric 3x3 A given as (xx, xy, xz, yy, yz, zz) plus
// s on the diagonal (adjugate over determinant; A is positive definite).
__device__ void solve_sym3(const double* a, double s, const double* b, double* x) {
  const double m00 = a[0] + s, m01 = a[1], m02 = a[2], m11 = a[3] + s, m12 = a[4], m22 = a[5] + s;
  const double c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
  const double c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
  const double det = m00 * c00 + m01 * c01 + m02 * c02;
  x[0] = (c00 * b[0] + c01 * b[1] + c02 * b[2]) / det;
  x[1] = (c01 * b[0] + c11 * b[1] + c12 * b[2]) / det;
  x[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) / det;
}

// ---------------------------------------------------------------------------
// k_colloid: colloid update ("molecular dynamics-like step", Sec. 2.2) and the
// end-of-step parity flip.  One block per box, one thread per colloid.  The
// velocity-dependent part of the link force is taken at the new velocity:
// V' = V + (M + zv)^{-1} (F_hyd + F_lc + F_ext), W' = W + (I + zw)^{-1} (T_hyd + T_lc + T_ext).
// ---------------------------------------------------------------------------
// Contact partner of colloid c at the current positions: -1 for a z wall,
// the lowest index of a colloid it touches, -2 for none.  The paper treats no
// contact (interactions between colloids are left to later work, Sec. 3.2);
// the reading taken: two colloids touch when their centres (minimum image)
// are closer than the sum of their radii, a colloid touches a wall when its
// surface passes the plane of the half-way bounce-back, z = -1/2 or nz - 1/2.
__device__ int contact_partner(const DevBox& B, int c) {
  const DevColloid& C = B.col[c];
  if (B.wall_z && (C.X[2] - C.a0 < -0.5 || C.X[2] + C.a0 > B.nz - 0.5)) return -1;
  for (int d = 0; d < B.ncol; ++d) {
    if (d == c) continue;
    double r[3];
    disp(B, C.X[0], C.X[1], C.X[2], B.col[d].X, r);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])), __dmul_rn(r[2], r[2]));
    const double s = __dadd_rn(C.a0, B.col[d].a0);
    if (r2 < __dmul_rn(s, s)) return d;
  }
  return -2;
}

// A mobile colloid whose new position touches a wall or another colloid is
// put back where it was before this step's move (its new velocities stand),
// so that no node is ever inside two colloids.  Every mobile colloid is tested
// at the same positions, then those in contact are put back; a colloid put
// back can be touched by another's move, so the test repeats until a pass
// puts none back.  The first contact since the host last read it (lowest
// colloid index of that pass) is kept in the box state and flagged in the
// group's error words; the host reports it as LC_ERR_OVERLAP.  All threads of
// the block call this (it holds block barriers).
__device__ void resolve_contacts(DevBox& B, int tid, int nthr) {
  __shared__ signed char s_hit[MAXCOL];  // -2 no contact, else the partner
  __shared__ unsigned char s_back[MAXCOL];
  __shared__ int s_any;
  for (int c = tid; c < B.ncol; c += nthr) s_back[c] = 0;
  for (int pass = 0; pass <= B.ncol; ++pass) {
    __syncthreads();
    for (int c = tid; c < B.ncol; c += nthr)
      s_hit[c] = (signed char)((B.col[c].mobile && !s_back[c]) ? contact_partner(B, c) : -2);
    if (tid == 0) s_any = 0;
    __syncthreads();
    for (int c = tid; c < B.ncol; c += nthr) {
      if (s_hit[c] == -2) continue;
      DevColloid& C = B.col[c];
      for (int a = 0; a < 3; ++a) C.X[a] = C.Xb[a];
      s_back[c] = 1;
      s_any = 1;
    }
    if (tid == 0) {
      DevState* st = B.st;
      for (int c = 0; c < B.ncol; ++c) {
        if (s_hit[c] == -2) continue;
        if (st->cstep < 0) {
          st->cstep = st->step;
          st->ccol = c;
          st->cpartner = s_hit[c];
        }
        st->err |= 8;
        atomicOr(B.gerr + 1, 1);
        break;
      }
    }
    __syncthreads();
    if (!s_any) break;
  }
}

template <bool CG>
__device__ __forceinline__ void colloid_box(DevBox& B, bool commit = true) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  if (!commit) {
    for (int c = tid; c < B.ncol; c += nthr)
      for (int k = 0; k < 24; ++k) B.col[c].acc[k] = 0.0;
    return;
  }
  for (int c = tid; c < B.ncol; c += nthr) {
    DevColloid& C = B.col[c];
    double acc[24];
    for (int k = 0; k < 24; ++k) acc[k] = CG ? __ldcg(&C.acc[k]) : C.acc[k];
    for (int a = 0; a < 3; ++a) {
      C.Fh[a] = acc[a];
      C.Th[a] = acc[3 + a];
      C.Flc[a] = acc[6 + a];
      C.Tlc[a] = acc[9 + a];
    }
    for (int a = 0; a < 3; ++a) {
      C.imp[a] += C.Fh[a] + C.Flc[a];
      C.aimp[a] += C.Th[a] + C.Tlc[a];
      C.Xb[a] = C.X[a];
      C.Vb[a] = C.V[a];
      C.Wb[a] = C.W[a];
    }
    if (C.mobile) {
      const double fv[3] = {C.Fh[0] + C.Flc[0] + C.Fext[0], C.Fh[1] + C.Flc[1] + C.Fext[1],
                            C.Fh[2] + C.Flc[2] + C.Fext[2]};
      const double tv[3] = {C.Th[0] + C.Tlc[0] + C.Text[0], C.Th[1] + C.Tlc[1] + C.Text[1],
                            C.Th[2] + C.Tlc[2] + C.Text[2]};
      double dv[3], dw[3];
      solve_sym3(acc + 12, C.M, fv, dv);
      solve_sym3(acc + 18, C.I, tv, dw);
      for (int a = 0; a < 3; ++a) {
        C.V[a] += dv[a];
        C.W[a] += dw[a];
      }
      const int L[3] = {B.nx, B.ny, B.nz};
      for (int a = 0; a < 3; ++a) {
        C.X[a] += C.V[a];
        if (a < 2 || !B.wall_z) {
          if (C.X[a] >= L[a]) C.X[a] -= L[a];
          if (C.X[a] < 0) C.X[a] += L[a];
        }
      }
    }
    for (int k = 0; k < 24; ++k) C.acc[k] = 0.0;
  }
  if (B.nmobile) resolve_contacts(B, tid, nthr);
  if (tid == 0) {
    DevState* st = B.st;
    if (B.p.flow_on) {
      st->fpar ^= 1;
      st->pre_valid = 0;
    }
    if (B.p.lc_on) st->qpar ^= 1;
    st->step += 1;
    st->nchg = 0;
  }
}

__global__ void k_colloid(DevBox* __restrict__ boxes, int nboxes) {
  const int b = blockIdx.x;
  if (b >= nboxes) return;
  colloid_box<false>(boxes[b]);
}

// ---------------------------------------------------------------------------
// k_step: one coupled step of every box as one persistent launch
// ---------------------------------------------------------------------------
// The blocks take work items in list order from an atomic counter.  The list
// is ordered so that every item comes after the items it waits for (stress of
// z chunks c - 1, c, c + 1 before the LB of chunk c; LB of c - 1, c, c + 1
// before the Q update of c; all LB tiles before the link exchange; all tiles
// and links before the colloid update), so the earliest unfinished item
// never waits on an item no block has taken, and the launch cannot deadlock
// whether or not all blocks are resident.  The phases of different chunks run
// side by side, so the HBM-bound LB overlaps the arithmetic-bound stress and
// Q update, and the stress, velocity and molecular field of a chunk are read
// back while they are still in L2.  Waits are bounded: after spin_limit
// polls the item is skipped (its outputs are then stale), *err is set and the
// host reports a timeout.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename T, int TY>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 ? 512 : 256) / (TX * TY)) k_step(
    DevBox* __restrict__ boxes, const StepItem* __restrict__ items, int nitems, int zc, unsigned* __restrict__ sync,
    double* __restrict__ part, int spin_limit, int commit, int* __restrict__ err) {
  __shared__ DevBox B;
  __shared__ double sblk[18];
  __shared__ int sq[TY][2 * TX];
  __shared__ int s_item, s_ok, s_sc0;
  const int tid = threadIdx.x + TX * threadIdx.y;
  int cur_box = -1;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(&sync[0], 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const StepItem I = items[it];
    if (tid == 0) {
      int ok = 1;
      for (int k = 0; k < 4 && ok; ++k) {
        if (I.wc[k] < 0) continue;
        const unsigned target = (unsigned)I.wt[k];
        for (int spin = 0; ld_acquire_u32(&sync[I.wc[k]]) < target; ++spin) {
          // give up after spin_limit polls, or at once when another wait of
          // this launch already gave up
          if (spin >= spin_limit || ((spin & 255) == 255 && ld_acquire_u32(reinterpret_cast<unsigned*>(err)) != 0)) {
            ok = 0;
            break;
          }
          __nanosleep(100);
        }
      }
      if (!ok) atomicOr(err, 1);
      s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
      load_box(B, boxes, I.box, cur_box);
      const int4 td = make_int4(I.box, I.x0, I.y0, I.z0);
      switch (I.kind) {
        case ITEM_STRESS:
          if constexpr (sizeof(T) == 4) {
            if (pair_box(B)) {
              stress_tile_pair<TY>(B, td, zc, FORCE_ACC, sq);
              break;
            }
          }
          stress_tile<T, TY>(B, td, zc, FORCE_ACC, sq);
          break;
        case ITEM_LB: lbp_tile<T, TY, true>(B, td, zc, sq); break;
        case ITEM_LC:
          if constexpr (sizeof(T) == 4) {
            if (pair_box(B)) {
              lc_tile_pair<TY, true>(B, td, zc, part + 2 * (size_t)I.part * TY, sq);
              break;
            }
          }
          lc_tile<T, TY, true>(B, td, zc, part + 2 * (size_t)I.part * TY, sq);
          break;
        case ITEM_LINKS: links_chunk<T, true>(B, I.x0, LINK_CHUNK, sblk, &s_sc0); break;
        default: colloid_box<true>(B, commit != 0); break;
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      if (I.dc[0] >= 0) atomicAdd(&sync[I.dc[0]], 1u);
      if (I.dc[1] >= 0) atomicAdd(&sync[I.dc[1]], 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// geometry: solid mask, near flags, boundary links (cold path)
// ---------------------------------------------------------------------------
__global__ void k_mask(DevBox* __restrict__ boxes, int b) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N) return;
  const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
  uint8_t id = 0;
  for (int c = 0; c < B.ncol; ++c)
    if (inside_colloid(B, x, y, z, B.col[c])) {
      if (id == 0) id = (uint8_t)(c + 1);
      else atomicOr(&B.st->err, 4);  // overlap
    }
  B.mask[i] = id;
}

__global__ void k_near(DevBox* __restrict__ boxes, int b) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N) return;
  uint8_t m = B.mask[i];
  if (m & IDMASK) return;
  const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
  bool near = false;
#pragma unroll
  for (int q = 1; q < NQ; ++q) {
    const int zz = z + cz(q);
    if (B.wall_z && (zz < 0 || zz >= B.nz)) {
      near = true;
      continue;
    }
    const int j = wrap1(x + cx(q), B.nx) + B.nx * (wrap1(y + cy(q), B.ny) + B.ny * wrap1(zz, B.nz));
    if (B.mask[j] & IDMASK) near = true;
  }
  B.mask[i] = near ? (uint8_t)(m | NEAR) : (uint8_t)(m & ~NEAR);
}

// Number of links from fluid node i into colloid c (bit q set in *bits).
__device__ __forceinline__ int links_at(const DevBox& B, int i, int c, unsigned* bits) {
  unsigned bm = 0;
  if ((B.mask[i] & IDMASK) == 0 && (B.mask[i] & NEAR)) {
    const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
#pragma unroll
    for (int q = 1; q < NQ; ++q) {
      const int zz = z + cz(q);
      if (B.wall_z && (zz < 0 || zz >= B.nz)) continue;
      const int j = wrap1(x + cx(q), B.nx) + B.nx * (wrap1(y + cy(q), B.ny) + B.ny * wrap1(zz, B.nz));
      if ((B.mask[j] & IDMASK) == (uint8_t)(c + 1)) bm |= 1u << q;
    }
  }
  *bits = bm;
  return __popc(bm);
}

__global__ void __launch_bounds__(256) k_link_count(const DevBox* __restrict__ boxes, int b, int c, int* blocksum) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned bits;
  int n = i < B.N ? links_at(B, i, c, &bits) : 0;
  __shared__ int s[8];
  int v = n;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < 8; ++k) t += s[k];
    blocksum[blockIdx.x] = t;
  }
}

// Exclusive scan of n ints in one block (deterministic); total -> *total.
__global__ void __launch_bounds__(1024) k_scan(int* a, int n, int base, int* total) {
  __shared__ int s[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = base;
  __syncthreads();
  for (int off = 0; off < n; off += 1024) {
    const int i = off + threadIdx.x;
    const int v = i < n ? a[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
      int t = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) a[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(256) k_link_write(const DevBox* __restrict__ boxes, int b, int c,
                                                    const int* blockoff) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned bits = 0;
  const int n = i < B.N ? links_at(B, i, c, &bits) : 0;
  __shared__ int s[256];
  s[threadIdx.x] = n;
  __syncthreads();
  for (int d = 1; d < 256; d <<= 1) {
    int t = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  int pos = blockoff[blockIdx.x] + s[threadIdx.x] - n;
  for (int q = 1; q < NQ; ++q)
    if (bits & (1u << q)) {
      if (pos < B.nlinks_cap) {
        B.link_node[pos] = i;
        B.link_dir[pos] = (int8_t)q;
        B.link_col[pos] = (int8_t)c;
      } else {
        atomicOr(&B.st->err, 1);
      }
      ++pos;
    }
}

// ---------------------------------------------------------------------------
// init, export, diagnostics (cold path)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t s) {
  uint64_t z = s + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Stores FP64 value v as component k of node i in both Q buffers (FP32:
// compensated, hi and its BF16 remainder).
template <typename T>
__device__ __forceinline__ void store_q(const DevBox& B, int i, int k, double v) {
  const size_t o = (size_t)k * B.N + i;
  if constexpr (sizeof(T) == 4) {
    float hi;
    __nv_bfloat16 lo;
    split_q(v, hi, lo);
    static_cast<float*>(B.Q[0])[o] = hi;
    static_cast<float*>(B.Q[1])[o] = hi;
    B.Qlo[0][o] = lo;
    B.Qlo[1][o] = lo;
  } else {
    static_cast<double*>(B.Q[0])[o] = v;
    static_cast<double*>(B.Q[1])[o] = v;
  }
}

// Stores FP64 value v as component k of node i of the current Q buffer only.
template <typename T>
__device__ __forceinline__ void store_q_cur(const DevBox& B, int i, int k, double v) {
  const int qpar = B.st->qpar;
  const size_t o = (size_t)k * B.N + i;
  if constexpr (sizeof(T) == 4) {
    float hi;
    __nv_bfloat16 lo;
    split_q(v, hi, lo);
    static_cast<float*>(B.Q[qpar])[o] = hi;
    B.Qlo[qpar][o] = lo;
  } else {
    static_cast<double*>(B.Q[qpar])[o] = v;
  }
}

// kind 0: uniaxial along (n0,n1,n2); kind 1: helix along axis (int)n0.
template <typename T>
__global__ void k_init_q(DevBox* __restrict__ boxes, int b, int kind, double n0, double n1, double n2, double amp,
                         unsigned long long seed) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N) return;
  const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
  double d[3];
  if (kind == 0) {
    const double nn = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(n0, n0), __dmul_rn(n1, n1)), __dmul_rn(n2, n2)));
    d[0] = n0 / nn; d[1] = n1 / nn; d[2] = n2 / nn;
  } else {
    const int ax = (int)n0, bb = (ax + 1) % 3, cc = (ax + 2) % 3;
    const int r[3] = {x, y, z};
    const double ph = B.p.q0 * r[ax];
    d[0] = d[1] = d[2] = 0.0;
    d[bb] = cos(ph);
    d[cc] = sin(ph);
  }
  // S0 (d_a d_b - delta_ab/3) with round-to-nearest operations only (no
  // contraction), so FP64 storage agrees bit for bit with a plain C evaluation.
  const double S0 = B.p.S0, third = 1.0 / 3.0;
  const double v[5] = {__dmul_rn(S0, __dsub_rn(__dmul_rn(d[0], d[0]), third)), __dmul_rn(S0, __dmul_rn(d[0], d[1])),
                       __dmul_rn(S0, __dmul_rn(d[0], d[2])), __dmul_rn(S0, __dsub_rn(__dmul_rn(d[1], d[1]), third)),
                       __dmul_rn(S0, __dmul_rn(d[1], d[2]))};
  for (int k = 0; k < 5; ++k) {
    const uint64_t r = splitmix64((uint64_t)seed ^ (uint64_t)(5LL * i + k));
    const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    const double val = __dadd_rn(v[k], __dmul_rn(amp, __dsub_rn(2.0 * u, 1.0)));
    store_q<T>(B, i, k, val);
  }
}

// Convert FP64 input to storage: which 0 = Q (both buffers), 1 = f (pre-collision,
// full f -> deviation into f[fpar], pre_valid set by the host).
template <typename T>
__global__ void k_set_field(DevBox* __restrict__ boxes, int b, int which, const double* __restrict__ src) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N) return;
  if (which == 0) {
    for (int k = 0; k < 5; ++k) store_q<T>(B, i, k, src[(size_t)k * B.N + i]);
  } else {
    T* f = static_cast<T*>(B.f[B.st->fpar]);
    for (int q = 0; q < NQ; ++q) f[(size_t)q * B.N + i] = T(src[(size_t)q * B.N + i] - wq(q) * B.p.rho0);
  }
}

// Exports.  which: LC_Q, LC_F_PRE, LC_RHO, LC_U, LC_FORCE, LC_SOLID.
template <typename T>
__global__ void k_export(const DevBox* __restrict__ boxes, int b, int which, double* __restrict__ out) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.N) return;
  const int N = B.N;
  const uint8_t m = B.mask[i];
  const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
  if (which == EXP_Q) {
    for (int k = 0; k < 5; ++k) out[(size_t)k * N + i] = load_q<T>(B, i, k);
    return;
  }
  if (which == EXP_SOLID) {
    out[i] = (m & IDMASK) ? (double)((m & IDMASK) - 1) : -1.0;
    return;
  }
  if (which == EXP_FORCE) {
    const T* F = static_cast<const T*>(B.F);
    for (int a = 0; a < 3; ++a) out[(size_t)a * N + i] = (m & IDMASK) || !B.p.lc_on ? 0.0 : (double)F[(size_t)a * N + i];
    return;
  }
  if (m & IDMASK) {
    if (which == EXP_F) {
      for (int q = 0; q < NQ; ++q) out[(size_t)q * N + i] = 0.0;
    } else if (which == EXP_RHO) {
      out[i] = B.p.rho0;
    } else {
      const DevColloid& C = B.col[(m & IDMASK) - 1];
      double d[3], ur[3];
      disp(B, (double)x, (double)y, (double)z, C.X, d);
      rigid_velocity(C.V, C.W, d, ur);
      for (int a = 0; a < 3; ++a) out[(size_t)a * N + i] = ur[a];
    }
    return;
  }
  T df[NQ];
  pull(B, static_cast<const T*>(B.f[B.st->fpar]), x, y, z, i, m, B.st->pre_valid != 0, df);
  if (which == EXP_F) {
    for (int q = 0; q < NQ; ++q) out[(size_t)q * N + i] = wq(q) * B.p.rho0 + (double)df[q];
    return;
  }
  double drho = 0.0, mm[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < NQ; ++q) {
    drho += (double)df[q];
    mm[0] += cx(q) * (double)df[q];
    mm[1] += cy(q) * (double)df[q];
    mm[2] += cz(q) * (double)df[q];
  }
  const double rho = B.p.rho0 + drho;
  if (which == EXP_RHO) {
    out[i] = rho;
    return;
  }
  const T* F = static_cast<const T*>(B.F);
  for (int a = 0; a < 3; ++a) {
    const double Fa = (B.p.lc_on ? (double)F[(size_t)a * N + i] : 0.0) + B.p.g[a];
    out[(size_t)a * N + i] = (mm[a] + 0.5 * Fa) / rho;
  }
}

// Diagnostics per block: [0] sum(df), [1..3] sum(df c), [4] fluid nodes,
// [5] defect nodes (3/2 lambda_max(Q) < 0.435).
template <typename T>
__global__ void __launch_bounds__(256) k_diag_state(const DevBox* __restrict__ boxes, int b, double* __restrict__ part) {
  const DevBox& B = boxes[b];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v[6] = {0, 0, 0, 0, 0, 0};
  __shared__ double sred[32 * 6];
  if (i < B.N) {
    const uint8_t m = B.mask[i];
    if (!(m & IDMASK)) {
      const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
      T df[NQ];
      pull(B, static_cast<const T*>(B.f[B.st->fpar]), x, y, z, i, m, B.st->pre_valid != 0, df);
      for (int q = 0; q < NQ; ++q) {
        v[0] += (double)df[q];
        v[1] += cx(q) * (double)df[q];
        v[2] += cy(q) * (double)df[q];
        v[3] += cz(q) * (double)df[q];
      }
      v[4] = 1.0;
      double q[5];
      for (int k = 0; k < 5; ++k) q[k] = load_q<T>(B, i, k);
      // largest eigenvalue of the traceless symmetric Q (closed form, as in principal_dir)
      double a00 = q[0], a01 = q[1], a02 = q[2], a11 = q[3], a12 = q[4], a22 = -q[0] - q[3];
      double p1 = a01 * a01 + a02 * a02 + a12 * a12;
      double p2 = a00 * a00 + a11 * a11 + a22 * a22 + 2.0 * p1;
      double lam = 0.0;
      if (p2 > 0.0) {
        double p = sqrt(p2 / 6.0);
        double b00 = a00 / p, b01 = a01 / p, b02 = a02 / p, b11 = a11 / p, b12 = a12 / p, b22 = a22 / p;
        double det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
        double r = fmin(1.0, fmax(-1.0, det / 2.0));
        lam = 2.0 * p * cos(acos(r) / 3.0);
      }
      v[5] = (1.5 * lam < 0.435) ? 1.0 : 0.0;
    }
  }
  block_sum<6>(v, sred);
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) part[6 * blockIdx.x + k] = v[k];
}

// Deterministic sum of n records of width w (column k) starting at rec0;
// out[k] = sum, or max for columns flagged in maxmask.
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ part, int rec0, int n, int w,
                                                unsigned maxmask, double* __restrict__ out) {
  __shared__ double s[256];
  for (int k = 0; k < w; ++k) {
    const bool ismax = (maxmask >> k) & 1u;
    double v = 0.0;
    for (int r = threadIdx.x; r < n; r += 256) {
      const double x = part[(size_t)(rec0 + r) * w + k];
      v = ismax ? fmax(v, x) : v + x;
    }
    s[threadIdx.x] = v;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
      if (threadIdx.x < d) s[threadIdx.x] = ismax ? fmax(s[threadIdx.x], s[threadIdx.x + d]) : s[threadIdx.x] + s[threadIdx.x + d];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = s[0];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// re-discretisation of moving colloids (Sec. 2.2, last paragraph)
// ---------------------------------------------------------------------------
// Run after the colloid update of every step for the (box, colloid) pairs of
// mobile colloids; every kernel returns at once when nothing changed.
//   k_rd_find     nodes of the colloid's bounding region whose solid test at
//                 the new X differs from the mask -> change list
//   k_rd_pull     pre-collision populations of the step just streamed, pulled
//                 with the old mask and the old colloid state, into the other
//                 buffer (the next collide reads them in place)
//   k_rd_apply    covered nodes hand their momentum sum_q df_q c_q to the
//                 colloid; uncovered nodes take f_eq(rho_bar, u_b) and the
//                 mean Q of their fluid face neighbours (fluid before and after)
//   k_rd_mask     mask bits of the changed nodes; k_rd_near the near flags of
//                 the region; k_rd_links the boundary links of the box.
__device__ __forceinline__ int region_lo(double c, double r) { return (int)floor(c - r - 2.0); }

// Node (x,y,z) of the bounding region of colloid C: index k of n = nx*ny*nz region
// nodes; returns false when the region node falls outside a z wall.
__device__ __forceinline__ bool region_node(const DevBox& B, const DevColloid& C, int k, int& x, int& y, int& z) {
  const int lx = region_lo(C.X[0], C.a0), ly = region_lo(C.X[1], C.a0), lz = region_lo(C.X[2], C.a0);
  const int ex = min(B.nx, (int)ceil(2.0 * C.a0) + 5), ey = min(B.ny, (int)ceil(2.0 * C.a0) + 5),
            ez = min(B.nz, (int)ceil(2.0 * C.a0) + 5);
  const int ix = k % ex, iy = (k / ex) % ey, iz = k / (ex * ey);
  x = wrapn(lx + ix, B.nx);
  y = wrapn(ly + iy, B.ny);
  z = lz + iz;
  if (B.wall_z) return z >= 0 && z < B.nz;
  z = wrapn(z, B.nz);
  return true;
}

__device__ __forceinline__ int region_size(const DevBox& B, const DevColloid& C) {
  const int e = (int)ceil(2.0 * C.a0) + 5;
  return min(B.nx, e) * min(B.ny, e) * min(B.nz, e);
}

// New solid owner of node (x,y,z): colloid index + 1, or 0.  No node is
// inside two colloids: add_colloid refuses a colloid that touches another and
// the colloid update puts back a move into contact (resolve_contacts), so the
// first colloid found is the only one.
__device__ __forceinline__ int new_owner(const DevBox& B, int x, int y, int z) {
  for (int c = 0; c < B.ncol; ++c)
    if (inside_colloid(B, x, y, z, B.col[c])) return c + 1;
  return 0;
}

__global__ void __launch_bounds__(256) k_rd_find(DevBox* __restrict__ boxes, const int2* __restrict__ mob, int nmob) {
  for (int p = blockIdx.y; p < nmob; p += gridDim.y) {
    const DevBox& B = boxes[mob[p].x];
    const DevColloid& C = B.col[mob[p].y];
    const int n = region_size(B, C);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
      int x, y, z;
      if (!region_node(B, C, k, x, y, z)) continue;
      const int i = x + B.nx * (y + B.ny * z);
      const int old = B.mask[i] & IDMASK;
      const bool in_new = inside_colloid(B, x, y, z, C);
      const int c = mob[p].y;
      int code = -1;
      if (in_new && old == 0) code = c << 1;                 // covered
      else if (!in_new && old == c + 1) code = (c << 1) | 1;  // uncovered
      else if (in_new && old != 0 && old != c + 1) atomicOr(&B.st->err, 4);
      if (code >= 0) {
        const int slot = atomicAdd(&B.st->nchg, 1);
        if (slot < B.chg_cap) {
          B.chg[2 * slot] = i;
          B.chg[2 * slot + 1] = code;
        } else {
          atomicOr(&B.st->err, 2);
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rd_pull(DevBox* __restrict__ boxes, int nboxes) {
  for (int b = 0; b < nboxes; ++b) {
    const DevBox& B = boxes[b];
    if (B.st->nchg == 0 || !B.p.flow_on) continue;
    const int fpar = B.st->fpar;
    const bool pre = B.st->pre_valid != 0;
    const T* fin = static_cast<const T*>(B.f[fpar]);
    T* fpre = static_cast<T*>(B.f[fpar ^ 1]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.N; i += gridDim.x * blockDim.x) {
      const uint8_t m = B.mask[i];
      if (m & IDMASK) continue;
      const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
      T df[NQ];
      pull(B, fin, x, y, z, i, m, pre, df);
#pragma unroll
      for (int q = 0; q < NQ; ++q) fpre[(size_t)q * B.N + i] = df[q];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rd_apply(DevBox* __restrict__ boxes, int nboxes) {
  for (int b = 0; b < nboxes; ++b) {
    DevBox& B = boxes[b];
    const int nchg = min(B.st->nchg, B.chg_cap);
    if (nchg == 0) continue;
    const int fpar = B.st->fpar;
    T* fpre = static_cast<T*>(B.f[fpar ^ 1]);
    const int N = B.N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nchg; k += gridDim.x * blockDim.x) {
      const int i = B.chg[2 * k], code = B.chg[2 * k + 1];
      const int c = code >> 1;
      DevColloid& C = B.col[c];
      const int x = i % B.nx, y = (i / B.nx) % B.ny, z = i / (B.nx * B.ny);
      if ((code & 1) == 0) {  // covered: its fluid momentum goes to the colloid
        if (B.p.flow_on) {
          double mom[3] = {0.0, 0.0, 0.0};
          for (int q = 0; q < NQ; ++q) {
            const double d = (double)fpre[(size_t)q * N + i];
            mom[0] += cx(q) * d;
            mom[1] += cy(q) * d;
            mom[2] += cz(q) * d;
            fpre[(size_t)q * N + i] = T(0);
          }
          for (int a = 0; a < 3; ++a) {
            atomicAdd(&C.imp[a], mom[a]);
            atomicAdd(&C.rdp[a], mom[a]);
          }
        }
        continue;
      }
      // uncovered: neighbours fluid before and after
      double rsum = 0.0, qsum[5] = {0, 0, 0, 0, 0};
      int cnt = 0;
      for (int d = 0; d < 6; ++d) {
        int xx = x, yy = y, zz = z;
        if (d == 0) xx = wrap1(x + 1, B.nx);
        if (d == 1) xx = wrap1(x - 1, B.nx);
        if (d == 2) yy = wrap1(y + 1, B.ny);
        if (d == 3) yy = wrap1(y - 1, B.ny);
        if (d == 4) zz = z + 1;
        if (d == 5) zz = z - 1;
        if (B.wall_z) {
          if (zz < 0 || zz >= B.nz) continue;
        } else {
          zz = wrap1(zz, B.nz);
        }
        const int j = xx + B.nx * (yy + B.ny * zz);
        if ((B.mask[j] & IDMASK) != 0 || new_owner(B, xx, yy, zz) != 0) continue;
        double rj = B.p.rho0;
        if (B.p.flow_on)
          for (int q = 0; q < NQ; ++q) rj += (double)fpre[(size_t)q * N + j];
        rsum += rj;
        for (int kk = 0; kk < 5; ++kk) qsum[kk] += load_q<T>(B, j, kk);
        ++cnt;
      }
      const double rb = cnt ? rsum / cnt : B.p.rho0;
      double dd[3], ubv[3];
      disp(B, (double)x, (double)y, (double)z, C.X, dd);
      rigid_velocity(C.V, C.W, dd, ubv);
      if (B.p.flow_on) {
        const double uu = ubv[0] * ubv[0] + ubv[1] * ubv[1] + ubv[2] * ubv[2];
        for (int q = 0; q < NQ; ++q) {
          const double cu = cx(q) * ubv[0] + cy(q) * ubv[1] + cz(q) * ubv[2];
          const double feq = wq(q) * rb * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
          fpre[(size_t)q * N + i] = T(feq - wq(q) * B.p.rho0);
        }
        for (int a = 0; a < 3; ++a) {
          atomicAdd(&C.imp[a], -rb * ubv[a]);
          atomicAdd(&C.rdp[a], -rb * ubv[a]);
        }
      }
      if (cnt)
        for (int kk = 0; kk < 5; ++kk) store_q_cur<T>(B, i, kk, qsum[kk] / cnt);
    }
  }
}

__global__ void __launch_bounds__(256) k_rd_mask(DevBox* __restrict__ boxes, int nboxes) {
  for (int b = 0; b < nboxes; ++b) {
    const DevBox& B = boxes[b];
    const int nchg = min(B.st->nchg, B.chg_cap);
    if (nchg == 0) continue;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nchg; k += gridDim.x * blockDim.x) {
      const int i = B.chg[2 * k], code = B.chg[2 * k + 1];
      B.mask[i] = (code & 1) ? (uint8_t)0 : (uint8_t)((code >> 1) + 1);
    }
  }
}

__global__ void __launch_bounds__(256) k_rd_near(DevBox* __restrict__ boxes, const int2* __restrict__ mob, int nmob) {
  for (int p = blockIdx.y; p < nmob; p += gridDim.y) {
    const DevBox& B = boxes[mob[p].x];
    if (B.st->nchg == 0) continue;
    const DevColloid& C = B.col[mob[p].y];
    const int n = region_size(B, C);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
      int x, y, z;
      if (!region_node(B, C, k, x, y, z)) continue;
      const int i = x + B.nx * (y + B.ny * z);
      const uint8_t m = B.mask[i];
      if (m & IDMASK) {
        B.mask[i] = m & IDMASK;
        continue;
      }
      bool near = false;
      for (int q = 1; q < NQ; ++q) {
        const int zz = z + cz(q);
        if (B.wall_z && (zz < 0 || zz >= B.nz)) {
          near = true;
          continue;
        }
        const int j = wrap1(x + cx(q), B.nx) + B.nx * (wrap1(y + cy(q), B.ny) + B.ny * wrap1(zz, B.nz));
        if (B.mask[j] & IDMASK) near = true;
      }
      B.mask[i] = near ? NEAR : (uint8_t)0;
    }
  }
}

// Rebuild the boundary links of boxes whose solid set changed (unordered;
// lc_lb_get_links sorts them).  Block 0 of the grid first clears the count
// in a separate launch (k_rd_links_reset).
__global__ void k_rd_links_reset(DevBox* __restrict__ boxes, int nboxes) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nboxes && boxes[b].st->nchg > 0) *boxes[b].nlinks = 0;
}

__global__ void __launch_bounds__(256) k_rd_links(DevBox* __restrict__ boxes, int nboxes) {
  for (int b = 0; b < nboxes; ++b) {
    const DevBox& B = boxes[b];
    if (B.st->nchg == 0) continue;
    for (int c = blockIdx.y; c < B.ncol; c += gridDim.y) {
      const DevColloid& C = B.col[c];
      const int n = region_size(B, C);
      for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int x, y, z;
        if (!region_node(B, C, k, x, y, z)) continue;
        const int i = x + B.nx * (y + B.ny * z);
        unsigned bits;
        const int nl = links_at(B, i, c, &bits);
        if (!nl) continue;
        int pos = atomicAdd(B.nlinks, nl);
        for (int q = 1; q < NQ; ++q)
          if (bits & (1u << q)) {
            if (pos < B.nlinks_cap) {
              B.link_node[pos] = i;
              B.link_dir[pos] = (int8_t)q;
              B.link_col[pos] = (int8_t)c;
            } else {
              atomicOr(&B.st->err, 1);
            }
            ++pos;
          }
      }
    }
  }
}

// The next collide reads the pulled populations in place; the momentum
// exchanged by the re-discretisation changes each mobile colloid's velocity.
__global__ void k_rd_finish(DevBox* __restrict__ boxes, int nboxes) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nboxes) return;
  DevBox& B = boxes[b];
  DevState* st = B.st;
  if (st->nchg == 0) return;
  if (B.p.flow_on) {
    st->fpar ^= 1;
    st->pre_valid = 1;
  }
  for (int c = 0; c < B.ncol; ++c) {
    DevColloid& C = B.col[c];
    if (C.mobile)
      for (int a = 0; a < 3; ++a) C.V[a] += C.rdp[a] / C.M;
    for (int a = 0; a < 3; ++a) C.rdp[a] = 0.0;
  }
  if (*B.nlinks > B.nlinks_cap) atomicOr(&st->err, 1);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename T, int TY>
static cudaError_t launch_force_t(const Launch& L, int mode, double* part) {
  constexpr int HP = (TX + 2) * (TY + 2);
  const size_t smem = sizeof(T) * 27 * HP + 3 * HP;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_force<T, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_force<T, TY><<<L.grid, dim3(TX, TY), smem, L.stream>>>(L.boxes, L.tiles, L.ntiles, L.zc, mode, part);
  return cudaGetLastError();
}

template <typename T, int TY>
static cudaError_t launch_lb_t(const Launch& L, int mode, double* part) {
  k_lb<T, TY><<<L.grid, dim3(TX, TY), 0, L.stream>>>(L.boxes, L.tiles, L.ntiles, L.zc, mode, part);
  return cudaGetLastError();
}

template <typename T, int BY>
static cudaError_t launch_flb_t(const Launch& L, int mode, double* part) {
  constexpr int HP = (TX + 2) * (BY + 2);
  const size_t smem = sizeof(T) * 27 * HP + 3 * HP;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_flb<T, BY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_flb<T, BY><<<L.grid, 32 * (BY + 3), smem, L.stream>>>(L.boxes, L.tiles, L.ntiles, L.zc, mode, part);
  return cudaGetLastError();
}

template <typename T, int TY>
static cudaError_t launch_stress_t(const Launch& L, int mode, double* part) {
  k_stress<T, TY><<<L.grid, dim3(TX, TY), 0, L.stream>>>(L.boxes, L.tiles, L.ntiles, L.zc, mode, part);
  return cudaGetLastError();
}

template <typename T, int TY>
static cudaError_t launch_lbp_t(const Launch& L, int mode, double* part) {
  k_lbp<T, TY><<<L.grid, dim3(TX, TY), 0, L.stream>>>(L.boxes, L.tiles, L.ntiles, L.zc, mode, part);
  return cudaGetLastError();
}

template <typename T, int TY>
static cudaError_t launch_lc_t(const Launch& L, int mode, double* part) {
  k_lc<T, TY><<<L.grid, dim3(TX, TY), 0, L.stream>>>(L.boxes, L.tiles, L.ntiles, L.zc, mode, part);
  return cudaGetLastError();
}

#define LCLB_DISPATCH_TY(FN, T)                      \
  switch (L.ty) {                                    \
    case 2: return FN<T, 2>(L, mode, part);          \
    case 4: return FN<T, 4>(L, mode, part);          \
    case 8: return FN<T, 8>(L, mode, part);          \
    default: return cudaErrorInvalidValue;           \
  }

cudaError_t launch_force(int prec, const Launch& L, int mode, double* part) {
  if (prec == 0) { LCLB_DISPATCH_TY(launch_force_t, float) }
  LCLB_DISPATCH_TY(launch_force_t, double)
}
cudaError_t launch_lb(int prec, const Launch& L, int mode, double* part) {
  if (prec == 0) { LCLB_DISPATCH_TY(launch_lb_t, float) }
  LCLB_DISPATCH_TY(launch_lb_t, double)
}
cudaError_t launch_flb(int prec, const Launch& L, int mode, double* part) {
  if (prec == 0) {
    switch (L.ty) {
      case 4: return launch_flb_t<float, 4>(L, mode, part);
      case 6: return launch_flb_t<float, 6>(L, mode, part);
      case 8: return launch_flb_t<float, 8>(L, mode, part);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (L.ty) {
    case 4: return launch_flb_t<double, 4>(L, mode, part);
    case 6: return launch_flb_t<double, 6>(L, mode, part);
    case 8: return launch_flb_t<double, 8>(L, mode, part);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t launch_lc(int prec, const Launch& L, int mode, double* part) {
  if (prec == 0) { LCLB_DISPATCH_TY(launch_lc_t, float) }
  LCLB_DISPATCH_TY(launch_lc_t, double)
}
cudaError_t launch_stress(int prec, const Launch& L, int mode, double* part) {
  if (prec == 0) { LCLB_DISPATCH_TY(launch_stress_t, float) }
  LCLB_DISPATCH_TY(launch_stress_t, double)
}
cudaError_t launch_lbp(int prec, const Launch& L, int mode, double* part) {
  if (prec == 0) { LCLB_DISPATCH_TY(launch_lbp_t, float) }
  LCLB_DISPATCH_TY(launch_lbp_t, double)
}

cudaError_t launch_links(int prec, const DevBox* boxes, const int2* chunks, int nchunks, int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  if (prec == 0) k_links<float><<<grid, 256, 0, s>>>(boxes, chunks, nchunks);
  else k_links<double><<<grid, 256, 0, s>>>(boxes, chunks, nchunks);
  return cudaGetLastError();
}

cudaError_t launch_colloid(DevBox* boxes, int nboxes, cudaStream_t s) {
  k_colloid<<<nboxes, 128, 0, s>>>(boxes, nboxes);
  return cudaGetLastError();
}

template <typename T, int TY>
static cudaError_t launch_step_t(DevBox* boxes, const StepItem* items, int nitems, int zc, unsigned* sync,
                                 double* part, int spin_limit, int commit, int* err, int grid, cudaStream_t s) {
  k_step<T, TY><<<grid, dim3(TX, TY), 0, s>>>(boxes, items, nitems, zc, sync, part, spin_limit, commit, err);
  return cudaGetLastError();
}

cudaError_t launch_step(int prec, int ty, DevBox* boxes, const StepItem* items, int nitems, int zc, unsigned* sync,
                        double* part, int spin_limit, int commit, int* err, int grid, cudaStream_t s) {
#define LCLB_STEP_CASE(T, Y) \
  case Y: return launch_step_t<T, Y>(boxes, items, nitems, zc, sync, part, spin_limit, commit, err, grid, s);
  if (prec == 0) {
    switch (ty) { LCLB_STEP_CASE(float, 2) LCLB_STEP_CASE(float, 4) LCLB_STEP_CASE(float, 8) default: break; }
  } else {
    switch (ty) { LCLB_STEP_CASE(double, 2) LCLB_STEP_CASE(double, 4) LCLB_STEP_CASE(double, 8) default: break; }
  }
#undef LCLB_STEP_CASE
  return cudaErrorInvalidValue;
}

int step_blocks_per_sm(int prec, int ty) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define LCLB_OCC(T, Y) \
  case Y: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<T, Y>, TX * Y, 0); break;
  if (prec == 0) {
    switch (ty) { LCLB_OCC(float, 2) LCLB_OCC(float, 4) LCLB_OCC(float, 8) default: break; }
  } else {
    switch (ty) { LCLB_OCC(double, 2) LCLB_OCC(double, 4) LCLB_OCC(double, 8) default: break; }
  }
#undef LCLB_OCC
  return e == cudaSuccess && n > 0 ? n : 1;
}

static inline int nblk(int N, int bs) { return (N + bs - 1) / bs; }

cudaError_t launch_geometry(DevBox* boxes, int b, int N, cudaStream_t s) {
  k_mask<<<nblk(N, 256), 256, 0, s>>>(boxes, b);
  k_near<<<nblk(N, 256), 256, 0, s>>>(boxes, b);
  return cudaGetLastError();
}

cudaError_t launch_link_build(DevBox* boxes, int b, int N, int c, int* blocksum, int base, int* total,
                              cudaStream_t s) {
  const int nb = nblk(N, 256);
  k_link_count<<<nb, 256, 0, s>>>(boxes, b, c, blocksum);
  k_scan<<<1, 1024, 0, s>>>(blocksum, nb, base, total);
  k_link_write<<<nb, 256, 0, s>>>(boxes, b, c, blocksum);
  return cudaGetLastError();
}

cudaError_t launch_init_q(int prec, DevBox* boxes, int b, int N, int kind, const double* n, double amp,
                          unsigned long long seed, cudaStream_t s) {
  if (prec == 0) k_init_q<float><<<nblk(N, 256), 256, 0, s>>>(boxes, b, kind, n[0], n[1], n[2], amp, seed);
  else k_init_q<double><<<nblk(N, 256), 256, 0, s>>>(boxes, b, kind, n[0], n[1], n[2], amp, seed);
  return cudaGetLastError();
}

cudaError_t launch_set_field(int prec, DevBox* boxes, int b, int N, int which, const double* src, cudaStream_t s) {
  if (prec == 0) k_set_field<float><<<nblk(N, 256), 256, 0, s>>>(boxes, b, which, src);
  else k_set_field<double><<<nblk(N, 256), 256, 0, s>>>(boxes, b, which, src);
  return cudaGetLastError();
}

cudaError_t launch_export(int prec, const DevBox* boxes, int b, int N, int which, double* out, cudaStream_t s) {
  if (prec == 0) k_export<float><<<nblk(N, 256), 256, 0, s>>>(boxes, b, which, out);
  else k_export<double><<<nblk(N, 256), 256, 0, s>>>(boxes, b, which, out);
  return cudaGetLastError();
}


cudaError_t launch_rediscretise(int prec, DevBox* boxes, int nboxes, const int2* mob, int nmob, int nsm,
                                cudaStream_t s) {
  if (nmob <= 0) return cudaSuccess;
  k_rd_find<<<dim3(8, nmob), 256, 0, s>>>(boxes, mob, nmob);
  if (prec == 0) k_rd_pull<float><<<nsm * 2, 256, 0, s>>>(boxes, nboxes);
  else k_rd_pull<double><<<nsm * 2, 256, 0, s>>>(boxes, nboxes);
  if (prec == 0) k_rd_apply<float><<<4, 256, 0, s>>>(boxes, nboxes);
  else k_rd_apply<double><<<4, 256, 0, s>>>(boxes, nboxes);
  k_rd_mask<<<4, 256, 0, s>>>(boxes, nboxes);
  k_rd_near<<<dim3(8, nmob), 256, 0, s>>>(boxes, mob, nmob);
  k_rd_links_reset<<<(nboxes + 127) / 128, 128, 0, s>>>(boxes, nboxes);
  k_rd_links<<<dim3(8, 4), 256, 0, s>>>(boxes, nboxes);
  k_rd_finish<<<(nboxes + 127) / 128, 128, 0, s>>>(boxes, nboxes);
  return cudaGetLastError();
}

int diag_state_blocks(int N) { return nblk(N, 256); }

cudaError_t launch_diag_state(int prec, const DevBox* boxes, int b, int N, double* part, cudaStream_t s) {
  if (prec == 0) k_diag_state<float><<<nblk(N, 256), 256, 0, s>>>(boxes, b, part);
  else k_diag_state<double><<<nblk(N, 256), 256, 0, s>>>(boxes, b, part);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* part, int rec0, int n, int w, unsigned maxmask, double* out, cudaStream_t s) {
  k_reduce<<<1, 256, 0, s>>>(part, rec0, n, w, maxmask, out);
  return cudaGetLastError();
}

}  // namespace lclb
