// lclb_dev.cuh -- device-side data structures and per-node physics of the
// hybrid LB / Beris-Edwards solver (Lintuvuori et al., Sec. 2).
//
// Storage: structure of arrays [component][z][y][x], node index
// x + nx*(y + ny*z).  Populations are stored as deviations df_i = f_i - w_i rho0
// after collision (pull scheme: the next step gathers df_i(r - c_i)).
// Q stores (xx, xy, xz, yy, yz); zz = -xx - yy.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lclb {

constexpr int NQ = 19;
constexpr int MAXCOL = 126;      // colloids per box (mask byte holds id + 1 in 7 bits)
constexpr uint8_t NEAR = 0x80;   // fluid node with a solid or wall node among its 18 neighbours
constexpr uint8_t IDMASK = 0x7F;
constexpr uint8_t WALLFLAG = 0xFF;  // "beyond a wall" marker in shared-memory flag planes

// D3Q19: rest; +x,-x,+y,-y,+z,-z; (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),
// (1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1); weights 1/3, 1/18, 1/36.
__host__ __device__ constexpr int cx(int q) {
  return q == 1 || q == 7 || q == 9 || q == 11 || q == 13 ? 1 : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int q) {
  return q == 3 || q == 7 || q == 10 || q == 15 || q == 17 ? 1 : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18 ? -1 : 0);
}
__host__ __device__ constexpr int cz(int q) {
  return q == 5 || q == 11 || q == 14 || q == 15 || q == 18 ? 1 : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr double wq(int q) { return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

struct DevParams {
  double rho0, tau, A0, gamma, K, q0, xi, Gamma, S0;
  double g[3];
  int lc_on, flow_on;
};

// The constants in the arithmetic type of the kernels (so that FP32 kernels
// never convert from FP64 per node).
template <typename T>
struct PhysT {
  T rho0, omega, pref;  // rho0, 1/tau, 1 - 1/(2 tau)
  T A0, gamma, K, q0, xi, Gamma, S0;
  T g[3];
};

// One colloid.  X, V, W: current state.  Xb, Vb, Wb: the state used when the
// post-collision populations now in memory were produced; the bounce-back of
// their streaming uses it.  acc: FP64 sums of the running step (F_hyd, T_hyd,
// F_lc, T_lc); Fh..Tlc: last completed step; imp/aimp: momentum received.
struct DevColloid {
  double X[3], V[3], W[3];
  double Xb[3], Vb[3], Wb[3];
  double a0, w, M, I;
  double Fext[3], Text[3];  // external force and torque
  int anchoring, mobile, strong, pad;
  double wfac;     // weight of Q0 in the surface value: w / (K + w), 1 for strong anchoring
  double acc[24];  // step sums: F_hyd, T_hyd, F_lc, T_lc, then the link drag tensors zv, zw (6 each, xx xy xz yy yz zz)
  double Fh[3], Th[3], Flc[3], Tlc[3];
  double imp[3], aimp[3];
  double rdp[3];  // momentum exchanged by the running re-discretisation
};

// Per-box state flags kept on the device (the step kernels flip the buffer
// parities without a host round trip).
struct DevState {
  int fpar;       // f[fpar] holds the current populations
  int qpar;       // Q[qpar] holds the current order parameter
  int pre_valid;  // f[fpar] holds pre-collision values: next collide reads them in place
  int err;        // sticky error bits (1: link list overflow, 2: change list overflow, 4: overlap, 8: contact)
  int nchg;       // nodes whose solid/fluid status changes after the colloid update of this step
  int pad;
  long long step;
  // first contact since the host last read it (see resolve_contacts): the
  // step, the colloid and its partner (-1: a z wall); cstep < 0: none
  long long cstep;
  int ccol, cpartner;
};

struct DevBox {
  int nx, ny, nz, wall_z;
  int pair;             // 1: FP32 box of even width (two-node paths of the stress kernel and the Q update)
  int nmobile;          // mobile colloids in the box (the colloid update tests contacts when > 0)
  int N, ncol;
  int nlinks_cap, chg_cap;
  int* chg;             // change list: (node, colloid << 1 | uncovered) pairs
  void* f[2];
  void* Q[2];
  // FP32 storage only (null for FP64): the BF16 remainder of each stored Q
  // component, so that hi + lo carries the increments that rounding hi alone
  // would drop (compensated storage; 5 comps, same layout as Q)
  __nv_bfloat16* Qlo[2];
  void* u;
  void* F;
  void* H;              // molecular field of the current Q at fluid nodes (5 comps), written by the stress kernels
  void* P;              // chemical stress at fluid nodes (9 comps, row-major P_ab), stored-stress variant only
  uint8_t* mask;
  DevColloid* col;
  DevState* st;
  int* gerr;            // error words of the box's group: [0] wait gave up, [1] contact in some box
  int* nlinks;          // device count of boundary links
  int* link_node;       // boundary links of this box, sorted by (colloid, node, dir)
  int8_t* link_dir;
  int8_t* link_col;
  DevParams p;
  PhysT<float> pf;
  PhysT<double> pd;
};

// FP32 boxes of even width run the two-node paths of the stress kernel and
// the Q update over tiles 64 nodes wide (those phases' tile lists step x by 64).
__host__ __device__ __forceinline__ bool pair_width(int nx, bool fp32) { return fp32 && nx % 2 == 0; }
__device__ __forceinline__ bool pair_box(const DevBox& B) { return B.pair != 0; }

template <typename T>
__device__ __forceinline__ const PhysT<T>& phys(const DevBox& B);
template <>
__device__ __forceinline__ const PhysT<float>& phys<float>(const DevBox& B) { return B.pf; }
template <>
__device__ __forceinline__ const PhysT<double>& phys<double>(const DevBox& B) { return B.pd; }

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int wrapn(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// Minimum-image displacement r - X along one axis (FP64, round-to-nearest
// operations only, matching a plain C evaluation).
__device__ __forceinline__ double minimg(double d, int L, bool periodic) {
  if (!periodic) return d;
  double h = 0.5 * (double)L;
  if (d >= h) d = __dsub_rn(d, (double)L);
  else if (d < -h) d = __dadd_rn(d, (double)L);
  return d;
}

__device__ __forceinline__ void disp(const DevBox& B, double x, double y, double z, const double* X, double d[3]) {
  d[0] = minimg(__dsub_rn(x, X[0]), B.nx, true);
  d[1] = minimg(__dsub_rn(y, X[1]), B.ny, true);
  d[2] = minimg(__dsub_rn(z, X[2]), B.nz, !B.wall_z);
}

// Solid test of Sec. 2.2: |r - X|^2 < a0^2, evaluated as dx*dx + dy*dy + dz*dz
// left to right with no fused multiply-add, so that it agrees bit for bit with
// a plain FP64 C evaluation.
__device__ __forceinline__ bool inside_colloid(const DevBox& B, int x, int y, int z, const DevColloid& C) {
  double d[3];
  disp(B, (double)x, (double)y, (double)z, C.X, d);
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return r2 < __dmul_rn(C.a0, C.a0);
}

// Compensated storage of Q in FP32: a value v (FP64) is kept as hi = RN32(v)
// and lo = RNbf16(v - hi); the stored value is hi + lo.
__device__ __forceinline__ void split_q(double v, float& hi, __nv_bfloat16& lo) {
  hi = (float)v;
  lo = __double2bfloat16(v - (double)hi);
}

// hi + lo + d carried into a new (hi, lo): the exact sum hi + s of
// s = lo + d by Knuth's branch-free two-sum (hi' = RN(hi + s) and the exact
// error of that addition), the error then rounded to BF16.
__device__ __forceinline__ void add_compensated(float hi, float lo, float d, float& hi_out, __nv_bfloat16& lo_out) {
  const float s = lo + d;
  const float h = __fadd_rn(hi, s);
  const float bb = __fsub_rn(h, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(h, bb)), __fsub_rn(s, bb));
  hi_out = h;
  lo_out = __float2bfloat16_rn(err);
}

// Stored value of component k of node i of the current Q (hi + lo for FP32).
template <typename T>
__device__ __forceinline__ double load_q(const DevBox& B, int i, int k) {
  const int qpar = B.st->qpar;
  const size_t o = (size_t)k * B.N + i;
  if constexpr (sizeof(T) == 4)
    return (double)static_cast<const float*>(B.Q[qpar])[o] + (double)__bfloat162float(B.Qlo[qpar][o]);
  else
    return static_cast<const double*>(B.Q[qpar])[o];
}

// Q entry (a,b) of the 5-component storage.
template <typename T>
__device__ __forceinline__ T qab(const T* q, int a, int b) {
  if (a > b) { int t = a; a = b; b = t; }
  if (a == 0) return b == 0 ? q[0] : (b == 1 ? q[1] : q[2]);
  if (a == 1) return b == 1 ? q[3] : q[4];
  return -q[0] - q[3];
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Minimum-image displacement and rigid velocity in the kernels' arithmetic
// type (used by the bounce-back of the LB kernel; the solid test itself is
// always FP64).
template <typename T>
__device__ __forceinline__ T minimg_t(T d, int L, bool periodic) {
  if (!periodic) return d;
  const T h = T(0.5) * T(L);
  if (d >= h) d -= T(L);
  else if (d < -h) d += T(L);
  return d;
}

template <typename T>
__device__ __forceinline__ void rigid_velocity_t(const DevBox& B, T x, T y, T z, const double* X, const double* V,
                                                 const double* W, T u[3]) {
  const T d0 = minimg_t(x - T(X[0]), B.nx, true);
  const T d1 = minimg_t(y - T(X[1]), B.ny, true);
  const T d2 = minimg_t(z - T(X[2]), B.nz, !B.wall_z);
  const T w0 = T(W[0]), w1 = T(W[1]), w2 = T(W[2]);
  u[0] = T(V[0]) + w1 * d2 - w2 * d1;
  u[1] = T(V[1]) + w2 * d0 - w0 * d2;
  u[2] = T(V[2]) + w0 * d1 - w1 * d0;
}

// Rigid-body velocity V + W x d.
__device__ __forceinline__ void rigid_velocity(const double* V, const double* W, const double d[3], double u[3]) {
  u[0] = V[0] + W[1] * d[2] - W[2] * d[1];
  u[1] = V[1] + W[2] * d[0] - W[0] * d[2];
  u[2] = V[2] + W[0] * d[1] - W[1] * d[0];
}

// Principal eigenvector of a symmetric traceless 3x3 matrix (5-component
// storage), from the closed-form trigonometric eigenvalue of a symmetric 3x3
// matrix (Smith, CACM 1961) and a cross product of two rows of (A - l I).
// FP64: the eigenvalue of the FP32 evaluation refined by two Newton steps on
// the characteristic polynomial det(A - l I) = -l^3 + (Tr A^2 / 2) l + det A
// (no FP64 transcendental functions), then the FP64 cross products.
template <typename T>
__device__ void principal_dir(const T* q, T n[3]);

__device__ __forceinline__ double principal_lambda_f64(const double* q) {
  const double a00 = q[0], a01 = q[1], a02 = q[2], a11 = q[3], a12 = q[4], a22 = -q[0] - q[3];
  const float qf[5] = {(float)q[0], (float)q[1], (float)q[2], (float)q[3], (float)q[4]};
  // FP32 seed: the largest eigenvalue by the trigonometric formula
  const float f00 = qf[0], f01 = qf[1], f02 = qf[2], f11 = qf[3], f12 = qf[4], f22 = -qf[0] - qf[3];
  const float p1 = f01 * f01 + f02 * f02 + f12 * f12;
  const float p2 = f00 * f00 + f11 * f11 + f22 * f22 + 2.f * p1;
  float lam32 = 0.f;
  if (p2 > 0.f) {
    const float pp = sqrtf(p2 / 6.f);
    const float b00 = f00 / pp, b01 = f01 / pp, b02 = f02 / pp, b11 = f11 / pp, b12 = f12 / pp, b22 = f22 / pp;
    float r = (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02)) / 2.f;
    r = fminf(1.f, fmaxf(-1.f, r));
    lam32 = 2.f * pp * cosf(acosf(r) / 3.f);
  }
  const double t2 = 0.5 * (a00 * a00 + a11 * a11 + a22 * a22 + 2.0 * (a01 * a01 + a02 * a02 + a12 * a12));
  const double det = a00 * (a11 * a22 - a12 * a12) - a01 * (a01 * a22 - a12 * a02) + a02 * (a01 * a12 - a11 * a02);
  double lam = (double)lam32;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double f = -lam * lam * lam + t2 * lam + det;
    const double df = -3.0 * lam * lam + t2;
    if (df != 0.0) lam -= f / df;
  }
  return lam;
}

template <typename T>
__device__ void principal_dir(const T* q, T n[3]) {
  T a00 = q[0], a01 = q[1], a02 = q[2], a11 = q[3], a12 = q[4], a22 = -q[0] - q[3];
  T p1 = a01 * a01 + a02 * a02 + a12 * a12;
  T p2 = a00 * a00 + a11 * a11 + a22 * a22 + T(2) * p1;
  if (!(p2 > T(0))) {
    n[0] = T(1); n[1] = T(0); n[2] = T(0);
    return;
  }
  T lam;
  if constexpr (sizeof(T) == 8) {
    lam = principal_lambda_f64(q);
  } else {
    T p = sqrt(p2 / T(6));
    T b00 = a00 / p, b01 = a01 / p, b02 = a02 / p, b11 = a11 / p, b12 = a12 / p, b22 = a22 / p;
    T det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
    T r = det / T(2);
    r = r < T(-1) ? T(-1) : (r > T(1) ? T(1) : r);
    T phi = acos(r) / T(3);
    lam = T(2) * p * cos(phi);
  }
  T r0[3] = {a00 - lam, a01, a02}, r1[3] = {a01, a11 - lam, a12}, r2[3] = {a02, a12, a22 - lam};
  T c0[3] = {r0[1] * r1[2] - r0[2] * r1[1], r0[2] * r1[0] - r0[0] * r1[2], r0[0] * r1[1] - r0[1] * r1[0]};
  T c1[3] = {r0[1] * r2[2] - r0[2] * r2[1], r0[2] * r2[0] - r0[0] * r2[2], r0[0] * r2[1] - r0[1] * r2[0]};
  T c2[3] = {r1[1] * r2[2] - r1[2] * r2[1], r1[2] * r2[0] - r1[0] * r2[2], r1[0] * r2[1] - r1[1] * r2[0]};
  T n0 = c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2];
  T n1 = c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2];
  T n2 = c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2];
  const T* c = c0;
  T nn = n0;
  if (n1 > nn) { c = c1; nn = n1; }
  if (n2 > nn) { c = c2; nn = n2; }
  if (!(nn > T(0))) {
    n[0] = T(1); n[1] = T(0); n[2] = T(0);
    return;
  }
  T s = T(1) / sqrt(nn);
  n[0] = c[0] * s; n[1] = c[1] * s; n[2] = c[2] * s;
}

// Surface order Q0 = S0 (n0 n0 - delta/3) (Eq. 7) at solid node (sx,sy,sz) of
// colloid c (c < 0: a z wall, homeotropic along z).  Homeotropic: n0 = unit
// normal s at the solid node; planar: n0 = projection of the fluid node's
// director (principal eigenvector of qf) on the plane normal to s.
template <typename T>
__device__ void surface_q0(const DevBox& B, int c, int sx, int sy, int sz, const T* qf, T q0[5]) {
  T n[3];
  if (c < 0) {
    n[0] = T(0); n[1] = T(0); n[2] = T(1);
  } else {
    const DevColloid& C = B.col[c];
    // the normal only orients Q0: the minimum-image offset is taken in FP64
    // (positions up to the box size), its normalisation in T
    double dd[3];
    disp(B, (double)sx, (double)sy, (double)sz, C.X, dd);
    const T d0 = T(dd[0]), d1 = T(dd[1]), d2 = T(dd[2]);
    const T r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    T s[3] = {d0 / r, d1 / r, d2 / r};
    if (C.anchoring == 0) {
      n[0] = s[0]; n[1] = s[1]; n[2] = s[2];
    } else {
      T nf[3];
      principal_dir(qf, nf);
      T ns = nf[0] * s[0] + nf[1] * s[1] + nf[2] * s[2];
      T p[3] = {nf[0] - ns * s[0], nf[1] - ns * s[1], nf[2] - ns * s[2]};
      T pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
      const T tiny = sizeof(T) == 8 ? T(1e-12) : T(1e-6);
      if (pn < tiny) {  // director along the normal: tangent s x e_k, k least aligned with s
        int k = 0;
        if (fabs(s[1]) < fabs(s[k])) k = 1;
        if (fabs(s[2]) < fabs(s[k])) k = 2;
        T e[3] = {T(0), T(0), T(0)};
        e[k] = T(1);
        p[0] = s[1] * e[2] - s[2] * e[1];
        p[1] = s[2] * e[0] - s[0] * e[2];
        p[2] = s[0] * e[1] - s[1] * e[0];
        pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
      }
      n[0] = p[0] / pn; n[1] = p[1] / pn; n[2] = p[2] / pn;
    }
  }
  T S0 = phys<T>(B).S0;
  T third = T(1) / T(3);
  q0[0] = S0 * (n[0] * n[0] - third);
  q0[1] = S0 * n[0] * n[1];
  q0[2] = S0 * n[0] * n[2];
  q0[3] = S0 * (n[1] * n[1] - third);
  q0[4] = S0 * n[1] * n[2];
}

// Value standing in for a solid (or wall) neighbour of a fluid node in the
// finite-difference stencil.  Strong anchoring: Q0.  Finite strength w: the
// minimiser of (w/2)|Qs - Q0|^2 + (K/2)|Qs - qf|^2, (K qf + w Q0)/(K + w).
// surf (if non-null) accumulates (w/2)|Qs - Q0|^2 (9 entries).
template <typename T>
__device__ void ghost_q(const DevBox& B, int c, int sx, int sy, int sz, const T* qf, T qs[5], double* surf) {
  T q0[5];
  surface_q0(B, c, sx, sy, sz, qf, q0);
  bool strong = (c < 0) || B.col[c].strong;
  if (strong) {
#pragma unroll
    for (int k = 0; k < 5; ++k) qs[k] = q0[k];
    return;
  }
  T w = T(B.col[c].w), K = phys<T>(B).K;
  T inv = T(1) / (K + w);
#pragma unroll
  for (int k = 0; k < 5; ++k) qs[k] = (K * qf[k] + w * q0[k]) * inv;
  if (surf) {
    double t = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double dd = (double)qab(qs, a, b) - (double)qab(q0, a, b);
        t += dd * dd;
      }
    *surf += 0.5 * (double)B.col[c].w * t;
  }
}

// Neighbour indices of node (x,y,z) along +x,-x,+y,-y,+z,-z; -1 beyond a wall.
__device__ __forceinline__ void face_neighbours(const DevBox& B, int x, int y, int z, int nb[6], int cz6[2]) {
  int nx = B.nx, ny = B.ny, nz = B.nz;
  int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
  int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
  int zp, zm;
  if (B.wall_z) {
    zp = z + 1 < nz ? z + 1 : -1;
    zm = z > 0 ? z - 1 : -1;
  } else {
    zp = z + 1 == nz ? 0 : z + 1;
    zm = z == 0 ? nz - 1 : z - 1;
  }
  int row = nx * (y + ny * z);
  nb[0] = xp + row;
  nb[1] = xm + row;
  nb[2] = x + nx * (yp + ny * z);
  nb[3] = x + nx * (ym + ny * z);
  nb[4] = zp < 0 ? -1 : x + nx * (y + ny * zp);
  nb[5] = zm < 0 ? -1 : x + nx * (y + ny * zm);
  cz6[0] = zp;
  cz6[1] = zm;
}

// Q at a fluid node and its six face neighbours (surface values for solid or
// wall neighbours).  Returns the centre in qi, neighbours in qn[6][5].
template <typename T>
__device__ __forceinline__ void gather_q(const DevBox& B, const T* __restrict__ Q, int x, int y, int z, int i,
                                         uint8_t m, T qi[5], T qn[6][5], double* surf) {
  const int N = B.N;
#pragma unroll
  for (int k = 0; k < 5; ++k) qi[k] = ldg(Q + (size_t)k * N + i);
  int nb[6], zz[2];
  face_neighbours(B, x, y, z, nb, zz);
  if (!(m & NEAR)) {
#pragma unroll
    for (int d = 0; d < 6; ++d)
#pragma unroll
      for (int k = 0; k < 5; ++k) qn[d][k] = ldg(Q + (size_t)k * N + nb[d]);
    return;
  }
  const int nx = B.nx, ny = B.ny;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    int j = nb[d];
    int c = -1;
    bool solid;
    if (j < 0) {
      solid = true;
    } else {
      uint8_t mj = B.mask[j] & IDMASK;
      solid = mj != 0;
      c = (int)mj - 1;
    }
    if (!solid) {
#pragma unroll
      for (int k = 0; k < 5; ++k) qn[d][k] = ldg(Q + (size_t)k * N + j);
    } else {
      int sx = x, sy = y, sz = z;
      if (d == 0) sx = x + 1 == nx ? 0 : x + 1;
      if (d == 1) sx = x == 0 ? nx - 1 : x - 1;
      if (d == 2) sy = y + 1 == ny ? 0 : y + 1;
      if (d == 3) sy = y == 0 ? ny - 1 : y - 1;
      if (d == 4) sz = zz[0];
      if (d == 5) sz = zz[1];
      ghost_q(B, c, sx, sy, sz, qi, qn[d], surf);
    }
  }
}

// 1/sqrt(v) in FP64 from the FP32 estimate and one Newton step (relative
// error ~1e-14 for the unit vectors of the surface values).
__device__ __forceinline__ double rsqrt_f64(double v) {
  double r = (double)rsqrtf((float)v);
  return r * (1.5 - 0.5 * v * r * r);
}

// Surface order Q0 (Eq. 7) for the nodes next to a solid in FP32 storage, in
// FP64: the unit normal s at solid node (sx, sy, sz) of colloid c (c < 0: a z
// wall, n0 = z); homeotropic n0 = s, planar n0 = nf projected on the plane
// normal to s (nf: the node's director, computed once per node), the
// tie-break s x e_k as surface_q0.
__device__ __forceinline__ void surface_q0_near(const DevBox& B, int c, int sx, int sy, int sz, const double nf[3],
                                                double q0[5]) {
  double n[3];
  if (c < 0) {
    n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
  } else {
    const DevColloid& C = B.col[c];
    double d[3];
    disp(B, (double)sx, (double)sy, (double)sz, C.X, d);
    const double ri = rsqrt_f64(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double sv[3] = {d[0] * ri, d[1] * ri, d[2] * ri};
    if (C.anchoring == 0) {
      n[0] = sv[0]; n[1] = sv[1]; n[2] = sv[2];
    } else {
      const double ns = nf[0] * sv[0] + nf[1] * sv[1] + nf[2] * sv[2];
      double pv[3] = {nf[0] - ns * sv[0], nf[1] - ns * sv[1], nf[2] - ns * sv[2]};
      double p2 = pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2];
      if (p2 < 1e-24) {  // director along the normal: tangent s x e_k, k least aligned with s
        int k = 0;
        if (fabs(sv[1]) < fabs(sv[k])) k = 1;
        if (fabs(sv[2]) < fabs(sv[k])) k = 2;
        double e[3] = {0.0, 0.0, 0.0};
        e[k] = 1.0;
        pv[0] = sv[1] * e[2] - sv[2] * e[1];
        pv[1] = sv[2] * e[0] - sv[0] * e[2];
        pv[2] = sv[0] * e[1] - sv[1] * e[0];
        p2 = pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2];
      }
      const double pi = rsqrt_f64(p2);
      n[0] = pv[0] * pi; n[1] = pv[1] * pi; n[2] = pv[2] * pi;
    }
  }
  const double S0 = B.pd.S0, third = 1.0 / 3.0;
  q0[0] = S0 * (n[0] * n[0] - third);
  q0[1] = S0 * n[0] * n[1];
  q0[2] = S0 * n[0] * n[2];
  q0[3] = S0 * (n[1] * n[1] - third);
  q0[4] = S0 * n[1] * n[2];
}

// FP32 storage, node next to a solid or wall: the derivatives from the
// compensated values hi + lo of the node and of its face neighbours, each
// neighbour difference formed as (hi_j - hi_i) + (lo_j - lo_i), and a solid
// or wall neighbour's surface value as Q0 - Q_i scaled by w/(K + w) (1 for
// strong anchoring), with Q0 and that difference in FP64.  With hi alone the
// rounding of Q (~3e-8) enters the Laplacian of every node at the colloid
// surface, and the colloid's LC force, a small sum of large face terms, would
// carry it at ~1e-4 relative.  qi receives the node's Q (hi + lo in FP32).
__device__ __forceinline__ void near_derivatives_f32(const DevBox& B, int x, int y, int z, int i, float qi[5],
                                                     float dq[3][5], float lap[5]) {
  const int N = B.N, qpar = B.st->qpar;
  const float* __restrict__ Q = static_cast<const float*>(B.Q[qpar]);
  const __nv_bfloat16* __restrict__ Lo = B.Qlo[qpar];
  float qh[5], ql[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    qh[k] = __ldg(Q + (size_t)k * N + i);
    ql[k] = __bfloat162float(Lo[(size_t)k * N + i]);
    qi[k] = qh[k] + ql[k];
  }
  int nb[6], zz[2], cf[6];
  face_neighbours(B, x, y, z, nb, zz);
  const int nx = B.nx, ny = B.ny;
  bool planar = false;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int j = nb[d];
    cf[d] = j < 0 ? -1 : (int)(B.mask[j] & IDMASK) - 1;  // colloid of a solid neighbour, else -1
    if (cf[d] >= 0 && B.col[cf[d]].anchoring != 0) planar = true;
  }
  double nf[3] = {1.0, 0.0, 0.0};
  if (planar) {
    double qid[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) qid[k] = (double)qh[k] + (double)ql[k];
    principal_dir<double>(qid, nf);
  }
  float dn[6][5];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int j = nb[d];
    if (j >= 0 && cf[d] < 0) {
#pragma unroll
      for (int k = 0; k < 5; ++k)
        dn[d][k] = (__ldg(Q + (size_t)k * N + j) - qh[k]) + (__bfloat162float(Lo[(size_t)k * N + j]) - ql[k]);
    } else {
      int sx = x, sy = y, sz = z;
      if (d == 0) sx = x + 1 == nx ? 0 : x + 1;
      if (d == 1) sx = x == 0 ? nx - 1 : x - 1;
      if (d == 2) sy = y + 1 == ny ? 0 : y + 1;
      if (d == 3) sy = y == 0 ? ny - 1 : y - 1;
      if (d == 4) sz = zz[0];
      if (d == 5) sz = zz[1];
      const int c = j < 0 ? -1 : cf[d];
      double q0[5];
      surface_q0_near(B, c, sx, sy, sz, nf, q0);
      const double s = c < 0 ? 1.0 : B.col[c].wfac;
#pragma unroll
      for (int k = 0; k < 5; ++k) dn[d][k] = (float)(s * ((q0[k] - (double)qh[k]) - (double)ql[k]));
    }
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    dq[0][k] = 0.5f * (dn[0][k] - dn[1][k]);
    dq[1][k] = 0.5f * (dn[2][k] - dn[3][k]);
    dq[2][k] = 0.5f * (dn[4][k] - dn[5][k]);
    lap[k] = (dn[0][k] + dn[1][k]) + (dn[2][k] + dn[3][k]) + (dn[4][k] + dn[5][k]);
  }
}

// Derivatives from the face-neighbour values: central first differences
// dq[g][k] = d_g Q_k and the 7-point Laplacian (Sec. 2.2: one stencil at all
// fluid nodes, surface values standing in for solid neighbours).
template <typename T>
__device__ __forceinline__ void derivatives(const T qi[5], const T qn[6][5], T dq[3][5], T lap[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    dq[0][k] = T(0.5) * (qn[0][k] - qn[1][k]);
    dq[1][k] = T(0.5) * (qn[2][k] - qn[3][k]);
    dq[2][k] = T(0.5) * (qn[4][k] - qn[5][k]);
    lap[k] = (qn[0][k] + qn[1][k]) + (qn[2][k] + qn[3][k]) + (qn[4][k] + qn[5][k]) - T(6) * qi[k];
  }
}

// C_ab = eps_agd d_g Q_db (a "curl" of Q acting on the first index).
template <typename T>
__device__ __forceinline__ T curlq(const T dq[3][5], int a, int b) {
  int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
  return qab(dq[a1], a2, b) - qab(dq[a2], a1, b);
}

// Molecular field H = -dF/dQ + Tr(dF/dQ) I/3 (Eq. 2) of the free energy of
// Eq. 1:
//   H = -A0(1-g/3) Q + A0 g (Q.Q - Tr(Q^2)/3 I) - A0 g Tr(Q^2) Q + K lap Q
//       - 2 K q0 (C + C^T) - 4 K q0^2 Q,     C_ab = eps_agd d_g Q_db.
template <typename T>
__device__ __forceinline__ void molecular_field(const PhysT<T>& P, const T q[5], const T dq[3][5], const T lap[5],
                                                T h[5]) {
  const T A0 = P.A0, g = P.gamma, K = P.K, q0 = P.q0;
  T trq2 = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) trq2 += qab(q, a, b) * qab(q, a, b);
  const T cb = -A0 * (T(1) - g / T(3)) - A0 * g * trq2 - T(4) * K * q0 * q0;
  const int ia[5] = {0, 0, 0, 1, 1}, ib[5] = {0, 1, 2, 1, 2};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int a = ia[k], b = ib[k];
    T q2 = qab(q, a, 0) * qab(q, 0, b) + qab(q, a, 1) * qab(q, 1, b) + qab(q, a, 2) * qab(q, 2, b);
    if (a == b) q2 -= trq2 / T(3);
    T chi = curlq(dq, a, b) + curlq(dq, b, a);
    h[k] = cb * q[k] + A0 * g * q2 + K * lap[k] - T(2) * K * q0 * chi;
  }
}

// Free energy density f' (Eq. 1 up to a total divergence):
//   f_bulk + K/2 |dQ|^2 + 2 K q0 Q_ab C_ab + 2 K q0^2 Tr(Q^2).
template <typename T>
__device__ __forceinline__ T free_energy_density(const PhysT<T>& P, const T q[5], const T dq[3][5]) {
  const T A0 = P.A0, g = P.gamma, K = P.K, q0 = P.q0;
  T trq2 = T(0), trq3 = T(0), grad2 = T(0), chi = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T qv = qab(q, a, b);
      trq2 += qv * qv;
      trq3 += qv * (qab(q, b, 0) * qab(q, 0, a) + qab(q, b, 1) * qab(q, 1, a) + qab(q, b, 2) * qab(q, 2, a));
      chi += qv * curlq(dq, a, b);
#pragma unroll
      for (int gg = 0; gg < 3; ++gg) grad2 += qab(dq[gg], a, b) * qab(dq[gg], a, b);
    }
  T fb = T(0.5) * A0 * (T(1) - g / T(3)) * trq2 - A0 * g / T(3) * trq3 + T(0.25) * A0 * g * trq2 * trq2;
  return fb + T(0.5) * K * grad2 + T(2) * K * q0 * chi + T(2) * K * q0 * q0 * trq2;
}

// Stress of Eq. 4 with P0 = rho cs^2 - f' (the LB carries rho cs^2):
//   P_ab = f' d_ab + 2 xi (Q_ab + d_ab/3) Q:H - xi (A_ab + A_ba) - (2 xi/3) H_ab
//          - E_ab + A_ab - A_ba,        A = Q H,
//   E_ab = d_a Q_gn Pi_b,gn = K <d_a Q, d_b Q> + 2 K q0 sum_gn d_a Q_gn G^b_gn,
//   G^b_gn = eps_mbg Q_mn.
// p[3*a + b].
template <typename T>
__device__ __forceinline__ void stress(const PhysT<T>& P, const T q[5], const T dq[3][5], const T h[5], T fprime,
                                       T p[9]) {
  const T K = P.K, q0 = P.q0, xi = P.xi;
  T A[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      A[a][b] = qab(q, a, 0) * qab(h, 0, b) + qab(q, a, 1) * qab(h, 1, b) + qab(q, a, 2) * qab(h, 2, b);
  T qh = A[0][0] + A[1][1] + A[2][2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T e1 = T(0), e2 = T(0);
#pragma unroll
      for (int gg = 0; gg < 3; ++gg)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          T da = qab(dq[a], gg, n);
          e1 += da * qab(dq[b], gg, n);
          if (gg != b) {
            int m = 3 - b - gg;  // eps(m, b, gg) != 0
            T sgn = ((m - b + 3) % 3 == 2) ? T(1) : T(-1);  // eps(m,b,g) = +1 when (m,b,g) is cyclic
            e2 += da * sgn * qab(q, m, n);
          }
        }
      T v = -(K * e1 + T(2) * K * q0 * e2);
      T dlt = a == b ? T(1) : T(0);
      v += fprime * dlt + T(2) * xi * (qab(q, a, b) + dlt / T(3)) * qh - xi * (A[a][b] + A[b][a]) -
           T(2) * xi / T(3) * qab(h, a, b) + A[a][b] - A[b][a];
      p[3 * a + b] = v;
    }
}

// All liquid-crystal quantities of one fluid node from its Q and its face-
// neighbour values, sharing intermediates: Q.Q (for H and Tr Q^3), the curl
// C_ab = eps_agd d_g Q_db (for the chiral part of H and of f'), and
// <d_a Q, d_b Q> for the 6 symmetric pairs (its trace is |grad Q|^2).
//   H   = cb Q + A0 g (Q.Q - Tr(Q^2) I/3) + K lap Q - 2 K q0 (C + C^T),
//         cb = -A0(1 - g/3) - A0 g Tr(Q^2) - 4 K q0^2                       (Eqs. 1, 2)
//   f'  = A0/2 (1-g/3) Tr Q^2 - A0 g/3 Tr Q^3 + A0 g/4 (Tr Q^2)^2
//         + K/2 |grad Q|^2 + 2 K q0 Q:C + 2 K q0^2 Tr Q^2                    (Eq. 1)
//   P   = f' I + 2 xi (Q + I/3) Q:H - xi (A + A^T) - (2 xi/3) H - E + A - A^T,
//         A = Q H,  E_ab = K <d_a Q, d_b Q> + 2 K q0 sum_gn d_a Q_gn eps_mbg Q_mn  (Eq. 4)
// The same expressions as molecular_field / free_energy_density / stress.
// lc_node_d: the same from the derivatives dq[g][k] = d_g Q_k and the
// Laplacian lap[k].  T is the arithmetic type of the node values (float,
// double, or f2: two nodes at once); C that of the constants (float for f2).
// Every constant factor is formed in C first, so that for f2 each term is one
// packed multiply or fused multiply-add.
template <typename T, bool NEED_P, typename C>
__device__ __forceinline__ void lc_node_d(const PhysT<C>& P, const T qi[5], const T dq[3][5], const T lap[5], T h[5],
                                          T p[9], T* fprime);

template <typename T, bool NEED_P>
__device__ __forceinline__ void lc_node(const PhysT<T>& P, const T qi[5], const T qn[6][5], T h[5], T p[9],
                                        T* fprime) {
  T dq[3][5], lap[5];
  derivatives(qi, qn, dq, lap);
  lc_node_d<T, NEED_P, T>(P, qi, dq, lap, h, p, fprime);
}

template <typename T, bool NEED_P, typename C>
__device__ __forceinline__ void lc_node_d(const PhysT<C>& P, const T qi[5], const T dq[3][5], const T lap[5], T h[5],
                                          T p[9], T* fprime) {
  const C A0 = P.A0, g = P.gamma, K = P.K, q0 = P.q0, xi = P.xi;
  const C third = C(1) / C(3);
  const C A0g = A0 * g, twoKq0 = C(2) * K * q0;
  const C c_lin = -A0 * (C(1) - g * third) - C(4) * K * q0 * q0;  // H: coefficient of Q beyond -A0 g Tr(Q^2)
  const C A0g3 = A0g * third;
  // Q (3x3), D[g] = d_g Q (3x3 each) from the 5 stored components
  T Q[3][3], D[3][3][3], S2[3][3], Cm[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Q[a][b] = qab(qi, a, b);
#pragma unroll
      for (int gg = 0; gg < 3; ++gg) D[gg][a][b] = qab(dq[gg], a, b);
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      S2[a][b] = Q[a][0] * Q[0][b] + Q[a][1] * Q[1][b] + Q[a][2] * Q[2][b];
      S2[b][a] = S2[a][b];
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Cm[a][b] = D[(a + 1) % 3][(a + 2) % 3][b] - D[(a + 2) % 3][(a + 1) % 3][b];
  const T trq2 = S2[0][0] + S2[1][1] + S2[2][2];
  const T cb = c_lin - A0g * trq2;
  const T tq3 = A0g3 * trq2;
  T H[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      const int k = a == 0 ? b : (a == 1 ? 2 + b : 5);
      const T lp = k < 5 ? lap[k] : -(lap[0] + lap[3]);
      T v = cb * Q[a][b] + A0g * S2[a][b] + K * lp - twoKq0 * (Cm[a][b] + Cm[b][a]);
      if (a == b) v = v - tq3;
      H[a][b] = v;
      H[b][a] = v;
    }
  h[0] = H[0][0]; h[1] = H[0][1]; h[2] = H[0][2]; h[3] = H[1][1]; h[4] = H[1][2];
  if (!NEED_P) return;
  // E_ab = K d_aQ : d_bQ; both factors are symmetric and traceless, so the
  // double contraction over the 5 stored components is
  // A_xx B_xx + A_yy B_yy + A_zz B_zz + 2 (A_xy B_xy + A_xz B_xz + A_yz B_yz)
  // with A_zz = -(A_xx + A_yy)
  T E[3][3], tz[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) tz[a] = dq[a][0] + dq[a][3];
  const C twoK = C(2) * K;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      const T e = K * (dq[a][0] * dq[b][0] + dq[a][3] * dq[b][3] + tz[a] * tz[b]) +
                  twoK * (dq[a][1] * dq[b][1] + dq[a][2] * dq[b][2] + dq[a][4] * dq[b][4]);
      E[a][b] = e;
      E[b][a] = e;
    }
  const T Kgrad2 = E[0][0] + E[1][1] + E[2][2];  // K |grad Q|^2
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // the chiral part: sum over g != b of eps(m, b, g) d_a Q_g. . Q_m. (m = 3 - b - g);
      // eps(m, b, g) = +1 for g = b + 1, m = b + 2 and -1 for g = b + 2, m = b + 1 (mod 3)
      const int g1 = (b + 1) % 3, g2 = (b + 2) % 3;
      const T e2 = (D[a][g1][0] * Q[g2][0] + D[a][g1][1] * Q[g2][1] + D[a][g1][2] * Q[g2][2]) -
                   (D[a][g2][0] * Q[g1][0] + D[a][g2][1] * Q[g1][1] + D[a][g2][2] * Q[g1][2]);
      E[a][b] = E[a][b] + twoKq0 * e2;
    }
  T trq3 = T(0), qc = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      trq3 = trq3 + Q[a][b] * S2[a][b];
      qc = qc + Q[a][b] * Cm[a][b];
    }
  const C fb2 = C(0.5) * A0 * (C(1) - g * third), fb4 = C(0.25) * A0g;
  const T fp = (fb2 * trq2 - A0g3 * trq3) + fb4 * (trq2 * trq2) + C(0.5) * Kgrad2 + twoKq0 * qc +
               (C(2) * K * q0 * q0) * trq2;
  T Am[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Am[a][b] = Q[a][0] * H[0][b] + Q[a][1] * H[1][b] + Q[a][2] * H[2][b];
  const T qh = Am[0][0] + Am[1][1] + Am[2][2];
  const C twoxi = C(2) * xi, twoxi3 = twoxi * third;
  const T qh2 = twoxi * qh;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // 2 xi (Q + I/3) Q:H - xi (A + A^T) - (2 xi/3) H - E + A - A^T, plus f' on the diagonal
      T v = qh2 * Q[a][b] - xi * (Am[a][b] + Am[b][a]) - twoxi3 * H[a][b] - E[a][b] + (Am[a][b] - Am[b][a]);
      if (a == b) v = v + (fp + third * qh2);
      p[3 * a + b] = v;
    }
  *fprime = fp;
}

}  // namespace lclb
