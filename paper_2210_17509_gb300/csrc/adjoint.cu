// Hand-written reverse mode of the FP64 method-of-lines step.
//
// Pieces (each the transpose of a forward kernel of this library):
//   * face adjoint: per face, recompute the reconstruction, the two face
//     states and the HLLE flux, then propagate the flux adjoint
//     Fbar = (Lbar_c - Lbar_{c-1}) / dx back through HLLE, the 3+1 state
//     formulas (Eqs. 6-9, 12, signal speeds) and WENO5 / minmod into the six
//     stencil cells (FP64 atomics) and into Gamma;
//   * source adjoint (curved metric): per cell, the hand-written reverse of
//     the Eq. 13 source (the source is linear in T^{mu nu}; the reverse runs
//     through b^mu, W, h* and P* to the primitives and Gamma);
//   * con2prim adjoint: the recovery is the inverse of prim -> cons, so its
//     adjoint solves (dU/dP)^T x = Pbar (implicit function theorem) with
//     dU/dP from dual numbers; prim -> cons adjoint multiplies by (dU/dP)^T;
//   * ghost-fill adjoint: every ghost point's adjoint is added to its source
//     interior point;
//   * the RK step reverse (SSP RK2 / RK3): recompute the stages, then sweep
//     them backwards.
#include <cmath>

#include "recovery.cuh"
#include "rhs.cuh"

namespace grmhd {

// ------------------------------------------------------------ dual numbers
// Forward-mode number with N derivative lanes (for per-cell 8x8 Jacobians).
template <int N>
struct Dn {
  double v;
  double d[N];
  __device__ Dn() {}
  __device__ Dn(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
};
template <int N> __device__ __forceinline__ Dn<N> operator+(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator-(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator-(const Dn<N>& a) {
  Dn<N> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator/(const Dn<N>& a, const Dn<N>& b) {
  Dn<N> r; r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator*(double a, const Dn<N>& b) {
  Dn<N> r; r.v = a * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a * b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dn<N> operator*(const Dn<N>& a, double b) { return b * a; }
template <int N> __device__ __forceinline__ Dn<N>& operator+=(Dn<N>& a, const Dn<N>& b) { a = a + b; return a; }
template <int N> __device__ __forceinline__ Dn<N>& operator-=(Dn<N>& a, const Dn<N>& b) { a = a - b; return a; }
template <int N> __device__ __forceinline__ Dn<N> xsqrt(const Dn<N>& a) {
  Dn<N> r; r.v = sqrt(a.v);
  const double s = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
  return r;
}

typedef Dn<9> D9;  // lanes 0..7: primitives, lane 8: Gamma

// Packed index of the symmetric pair (i, j) in [xx, xy, xz, yy, yz, zz].
__device__ __forceinline__ int sym_index(int i, int j) {
  const int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

// Conserved vector of one primitive state (Eqs. 6-9), generic scalar.
template <class T>
__device__ __forceinline__ void cons_of_prim(const T pr[8], const double g[6], double sg, T gfac, T U[8]) {
  const T v[3] = {pr[1], pr[2], pr[3]};
  const T B[3] = {pr[5], pr[6], pr[7]};
  T vl[3], Bl[3];
  vl[0] = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
  vl[1] = g[1] * v[0] + g[3] * v[1] + g[4] * v[2];
  vl[2] = g[2] * v[0] + g[4] * v[1] + g[5] * v[2];
  Bl[0] = g[0] * B[0] + g[1] * B[1] + g[2] * B[2];
  Bl[1] = g[1] * B[0] + g[3] * B[1] + g[4] * B[2];
  Bl[2] = g[2] * B[0] + g[4] * B[1] + g[5] * B[2];
  const T v2 = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
  const T Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const T B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const T omv2 = T(1.0) - v2;
  const T iW = xsqrt(omv2);
  const T W = T(1.0) / iW;
  const T ab0 = W * Bv;
  const T b2 = B2 * omv2 + Bv * Bv;
  const T hs = pr[0] + gfac * pr[4] + b2;
  const T Ps = pr[4] + T(0.5) * b2;
  const T hW2 = hs * W * W;
  const T D = T(sg) * pr[0] * W;
#pragma unroll
  for (int i = 0; i < 3; ++i) U[1 + i] = T(sg) * (hW2 * vl[i] - ab0 * (Bl[i] * iW + ab0 * vl[i]));
  U[0] = D;
  U[4] = T(sg) * (hW2 - Ps - ab0 * ab0) - D;
#pragma unroll
  for (int i = 0; i < 3; ++i) U[5 + i] = T(sg) * B[i];
}

// J[i][j] = dU_i / dP_j (j < 8) and dU_i / dGamma (j = 8) at the cell c.
__device__ __forceinline__ void cons_jacobian(const DevGrid& g, const DevParams& p, const double* __restrict__ prim,
                                              const double* __restrict__ metric, long long c, double J[8][9]) {
  CellMetric m;
  cell_metric(metric, g.ncell, c, m);
  D9 pr[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    pr[q] = D9(__ldg(prim + q * g.ncell + c));
    pr[q].d[q] = 1.0;
  }
  D9 gf(p.gfac);
  gf.d[8] = -1.0 / ((p.gamma - 1.0) * (p.gamma - 1.0));  // d/dGamma of Gamma/(Gamma-1)
  D9 U[8];
  cons_of_prim<D9>(pr, m.g, m.sqrtg, gf, U);
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 9; ++j) J[i][j] = U[i].d[j];
}

// Solve A^T x = b in place (b becomes x) for A = dU/dP (8x8), using its
// block form: the conserved field is sqrt(gamma) B, so the rows of U^5..7
// are sqrt(gamma) times the unit rows of B and A = [[A11, A12], [0, sg I]].
// Then A11^T x1 = b1 (5x5, partial pivoting) and x2 = (b2 - A12^T x1) / sg.
// Everything is unrolled with compile-time indices (the row exchanges are
// selects), so the matrix stays in registers; the pivot search compares
// magnitudes on the integer pipe.
__device__ __forceinline__ bool solve_transposed8(const double J[8][9], double b[8]) {
  constexpr int N = 5;
  double a[N][N], ip[N];
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) a[r][c] = J[c][r];  // A11^T
#pragma unroll
  for (int c = 0; c < N; ++c) {
    int piv = c;
    uint32_t bh, bl;
    dwords(a[c][c], bh, bl);
    bh &= 0x7fffffffu;
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      uint32_t h, l;
      dwords(a[r][c], h, l);
      h &= 0x7fffffffu;
      if (h > bh || (h == bh && l > bl)) { bh = h; bl = l; piv = r; }
    }
    if ((bh | bl) == 0u || bh >= 0x7ff00000u) return false;  // zero pivot, or not finite
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      const bool sw = piv == r;
#pragma unroll
      for (int k = c; k < N; ++k) {
        const double t = a[c][k];
        a[c][k] = sw ? a[r][k] : t;
        a[r][k] = sw ? t : a[r][k];
      }
      const double t = b[c];
      b[c] = sw ? b[r] : t;
      b[r] = sw ? t : b[r];
    }
    ip[c] = 1.0 / a[c][c];
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      const double f = a[r][c] * ip[c];
#pragma unroll
      for (int k = c + 1; k < N; ++k) a[r][k] -= f * a[c][k];
      b[r] -= f * b[c];
    }
  }
#pragma unroll
  for (int r = N - 1; r >= 0; --r) {
    double s = b[r];
#pragma unroll
    for (int k = r + 1; k < N; ++k) s -= a[r][k] * b[k];
    b[r] = s * ip[r];
  }
  const double sg = J[5][5];
  if (!dgt0i(sg) || !dfinitei(sg)) return false;
  const double isg = 1.0 / sg;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double s = b[5 + k];
#pragma unroll
    for (int i = 0; i < N; ++i) s -= J[i][5 + k] * b[i];
    b[5 + k] = s * isg;
  }
  return true;
}

__device__ __forceinline__ void block_add_gamma(double v, double* gamma_bar) {
  // warp reduction, then one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(gamma_bar, v);
}

// GRMHD_DETERMINISTIC: the same sum in a fixed order.  Every warp's partial
// (reduced as above) goes to its slot, blockIdx * warps + warp; the block
// that finishes last, elected by a ticket counter (no block waits for
// another), sums the slots in slot order through a fixed tree and adds the
// total to *gamma_bar once, then resets the ticket for the next launch.
// The slots are the library's, so deterministic reverse calls on concurrent
// streams would share them; they are meant for one stream at a time.
// Grids are at most 152 x 32 blocks (blocks_for) of at most 256 threads.
constexpr int kDetSlots = 152 * 32 * 8;
__device__ double g_det_slots[kDetSlots];
__device__ unsigned int g_det_ticket;

__device__ __noinline__ void block_add_gamma_det(double v, double* gamma_bar) {
  __shared__ double red[256];
  __shared__ unsigned int last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int nw = blockDim.x >> 5;
  const int nslot = min((int)gridDim.x * nw, kDetSlots);
  const int slot = blockIdx.x * nw + (threadIdx.x >> 5);
  if ((threadIdx.x & 31) == 0 && slot < kDetSlots) g_det_slots[slot] = v;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&g_det_ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < nslot; i += blockDim.x) s += __ldcg(g_det_slots + i);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (red[0] != 0.0) *gamma_bar += red[0];
    g_det_ticket = 0u;
  }
}

// Called by every thread of the block, once, at the end of the kernel.
__device__ __forceinline__ void add_gamma(const DevParams& p, double v, double* gamma_bar) {
  if (p.flags & GRMHD_DETERMINISTIC) block_add_gamma_det(v, gamma_bar);
  else block_add_gamma(v, gamma_bar);
}

// ---------------------------------------------------- con2prim / prim2con
// cons_bar += (dU/dP)^{-T} prim_bar;  gamma_bar -= x . dU/dGamma   (interior)
__global__ void con2prim_adjoint_kernel(DevGrid g, DevParams p, const double* __restrict__ prim,
                                        const double* __restrict__ metric, const double* __restrict__ prim_bar,
                                        double* __restrict__ cons_bar, double* __restrict__ gamma_bar,
                                        int* __restrict__ singular) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double gb = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, t);
    double J[8][9];
    cons_jacobian(g, p, prim, metric, c, J);
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = prim_bar[q * g.ncell + c];
    if (!solve_transposed8(J, x)) {
      atomicAdd(singular, 1);
      continue;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      cons_bar[q * g.ncell + c] += x[q];
      gb -= x[q] * J[q][8];
    }
  }
  add_gamma(p, gb, gamma_bar);
}

// prim_bar += (dU/dP)^T cons_bar;  gamma_bar += cons_bar . dU/dGamma   (interior)
__global__ void prim2con_adjoint_kernel(DevGrid g, DevParams p, const double* __restrict__ prim,
                                        const double* __restrict__ metric, const double* __restrict__ cons_bar,
                                        double* __restrict__ prim_bar, double* __restrict__ gamma_bar) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double gb = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, t);
    double J[8][9];
    cons_jacobian(g, p, prim, metric, c, J);
    double ub[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ub[q] = cons_bar[q * g.ncell + c];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < 8; ++i) s += J[i][j] * ub[i];
      prim_bar[j * g.ncell + c] += s;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) gb += ub[i] * J[i][8];
  }
  add_gamma(p, gb, gamma_bar);
}

// ------------------------------------------------------------ ghost fill
// Transpose of the ghost fill: each interior point gathers the adjoints of
// all ghost points that copy from it; ghost entries are then zero.
__global__ void fill_ghosts_adjoint_kernel(DevGrid g, int bc, int nvar, double* __restrict__ f) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    idx[0] = (int)(t % g.n[0]);
    idx[1] = (int)((t / g.n[0]) % g.n[1]);
    idx[2] = (int)(t / ((long long)g.n[0] * g.n[1]));
    // only interior points that some ghost copies from have work (copy:
    // the first and last point of an axis; periodic: the ng points at each
    // end, all of them on axes shorter than 2 ng); for the others the
    // gather below would store the point's own value back
    bool source = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int i = idx[d];
      source = source || (bc == GRMHD_BC_PERIODIC ? (i < g.ng || i >= g.n[d] - g.ng) : (i == 0 || i == g.n[d] - 1));
    }
    if (!source) continue;
    // per axis, every full-array coordinate whose source is this interior coordinate
    int pos[3][1 + 2 * 16];
    int cnt[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int i = idx[d];
      cnt[d] = 0;
      pos[d][cnt[d]++] = i + g.ng;
      for (int gpos = 0; gpos < g.ng; ++gpos) {
        const int lo = gpos - g.ng;        // interior-relative coordinate of a low ghost
        const int hi = g.n[d] + gpos;      // ... of a high ghost
        int slo, shi;
        if (bc == GRMHD_BC_PERIODIC) {
          slo = ((lo % g.n[d]) + g.n[d]) % g.n[d];
          shi = hi % g.n[d];
        } else {
          slo = 0;
          shi = g.n[d] - 1;
        }
        if (slo == i) pos[d][cnt[d]++] = lo + g.ng;
        if (shi == i) pos[d][cnt[d]++] = hi + g.ng;
      }
    }
    const long long self = (long long)(idx[2] + g.ng) * g.sz + (long long)(idx[1] + g.ng) * g.sy + (idx[0] + g.ng);
    for (int q = 0; q < nvar; ++q) {
      double s = 0.0;
      for (int a = 0; a < cnt[2]; ++a)
        for (int b = 0; b < cnt[1]; ++b)
          for (int e = 0; e < cnt[0]; ++e) {
            const long long cc = (long long)pos[2][a] * g.sz + (long long)pos[1][b] * g.sy + pos[0][e];
            s += f[q * g.ncell + cc];
            if (cc != self) f[q * g.ncell + cc] = 0.0;
          }
      f[q * g.ncell + self] = s;
    }
  }
}

// ----------------------------------------------------- reconstruction adjoint
// WENO5 value v(u0..u4) at the right face of the middle cell and its five
// partial derivatives dv/du_k, with the weights of the forward (indicators
// scaled by 12/13, product form; see weno5_cell_parts):
//   dv = sum_k o_k dq_k - 2 sum_k o_k (q_k - v) de_k / e_k.
// Everything before the two reciprocals 1/sum(w) and 1/(e0 e1 e2):
struct Weno5VG {
  double q[3];  // 6 q_k
  double t[3], s[3], e[3], p[3];  // p = (e1 e2, e0 e2, e0 e1)
  double w[3], ws, ee;            // weights, their sum, e0 e1 e2
};

__device__ __forceinline__ void weno5_vg_parts(const double u[5], double eps13, Weno5VG& a) {
  const double k313 = 3.0 / 13.0;
  a.q[0] = fma(2.0, u[0], fma(-7.0, u[1], 11.0 * u[2]));
  a.q[1] = fma(2.0, u[3], fma(5.0, u[2], -u[1]));
  a.q[2] = fma(5.0, u[3], fma(2.0, u[2], -u[4]));
  a.t[0] = fma(-2.0, u[1], u[0] + u[2]);
  a.s[0] = fma(3.0, u[2], fma(-4.0, u[1], u[0]));
  a.t[1] = fma(-2.0, u[2], u[1] + u[3]);
  a.s[1] = u[1] - u[3];
  a.t[2] = fma(-2.0, u[3], u[2] + u[4]);
  a.s[2] = fma(3.0, u[2], fma(-4.0, u[3], u[4]));
#pragma unroll
  for (int k = 0; k < 3; ++k) a.e[k] = fma(a.t[k], a.t[k], fma(k313 * a.s[k], a.s[k], eps13));
  a.p[0] = a.e[1] * a.e[2];
  a.p[1] = a.e[0] * a.e[2];
  a.p[2] = a.e[0] * a.e[1];
  a.w[0] = a.p[0] * a.p[0];
  a.w[1] = 6.0 * (a.p[1] * a.p[1]);
  a.w[2] = 3.0 * (a.p[2] * a.p[2]);
  a.ws = a.w[0] + a.w[1] + a.w[2];
  a.ee = a.e[0] * a.p[0];
}

// Value and gradient from the parts and the reciprocals iws = 1/ws, iee = 1/ee.
__device__ __forceinline__ double weno5_vg_finish(const Weno5VG& a, double iws, double iee, double gr[5]) {
  const double c6 = 1.0 / 6.0, k313 = 3.0 / 13.0;
  double o[3], tb[3], sb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) o[k] = a.w[k] * iws;
  const double v6 = fma(o[0], a.q[0], fma(o[1], a.q[1], o[2] * a.q[2]));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // -2 o_k (q_k - v) / e_k, with q_k - v = (6 q_k - 6 v) / 6 and 1/e_k = p_k / ee
    const double eb = (-2.0 * c6) * o[k] * (a.q[k] - v6) * (a.p[k] * iee);
    tb[k] = 2.0 * a.t[k] * eb;
    sb[k] = (2.0 * k313) * a.s[k] * eb;
    o[k] *= c6;
  }
  gr[0] = 2.0 * o[0] + tb[0] + sb[0];
  gr[1] = -7.0 * o[0] - o[1] - 2.0 * tb[0] - 4.0 * sb[0] + tb[1] + sb[1];
  gr[2] = 11.0 * o[0] + 5.0 * o[1] + 2.0 * o[2] + tb[0] + 3.0 * sb[0] - 2.0 * tb[1] + tb[2] + 3.0 * sb[2];
  gr[3] = 2.0 * o[1] + 5.0 * o[2] + tb[1] - sb[1] - 2.0 * tb[2] - 4.0 * sb[2];
  gr[4] = -o[2] + tb[2] + sb[2];
  return v6 * c6;
}

// Values and gradients of two stencils (the two states of a face); the four
// reciprocals come from one division.
__device__ __forceinline__ void weno5_value_grad2(const double uA[5], const double uB[5], double eps13, double& vA,
                                                  double grA[5], double& vB, double grB[5]) {
  Weno5VG A, B;
  weno5_vg_parts(uA, eps13, A);
  weno5_vg_parts(uB, eps13, B);
  const double xa = A.ws * A.ee, xb = B.ws * B.ee;
  const double Z = rcp_nr(xa * xb);
  const double ra = xb * Z, rb = xa * Z;
  vA = weno5_vg_finish(A, A.ee * ra, A.ws * ra, grA);
  vB = weno5_vg_finish(B, B.ee * rb, B.ws * rb, grB);
}

// Both WENO5 states of one cell from its stencil u[0..4] = u_{i-2..i+2},
// with their partial derivatives: vp / gp (plus: the value at the upper face
// i+1/2, gp[k] = dvp/du_k) and vm / gm (minus: the value at the lower face,
// from the mirrored stencil, gm[k] = dvm/du_k).  The mirrored stencil has
// the same smoothness indicators in reverse order (t, e and p reversed, s
// reversed with its middle entry negated, which the squares drop), so they
// are formed once; the three reciprocals 1/ws+, 1/ws- and 1/(e0 e1 e2) come
// from one division.  The derivative of a state is
//   dv/du_j = sum_k o_k dq_k/du_j + sum_k c_k (2 t_k dt_k/du_j + (6/13) s_k ds_k/du_j),
//   c_k = -2 o_k (q_k - v) / e_k,  o_k = w_k / ws
// (the weights sum to one, so the derivative of the normalisation drops
// out); 2 t_k, (6/13) s_k and -2 p_k / (e0 e1 e2) = -2 / e_k are shared by
// the two states.
struct Weno5CellGradShared {
  double t2[3], s613[3], m2ie[3];  // 2 t_k, (6/13) s_k, -2 p_k / ee (plus-state order)
};

// Value and gradient of one state from its parts (a: the state's stencil
// order), the shared factors in that order (t2, s613, m2ie) and 1/ws.
__device__ __forceinline__ double weno5_state_grad(const Weno5VG& a, const double t2[3], const double s613[3],
                                                   const double m2ie[3], double iws, double gr[5]) {
  const double c6 = 1.0 / 6.0;
  double oc[3], tb[3], sb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) oc[k] = (a.w[k] * iws) * c6;  // o_k / 6
  // 6 v (a.q holds 6 q_k)
  const double v6 = 6.0 * fma(oc[0], a.q[0], fma(oc[1], a.q[1], oc[2] * a.q[2]));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // c_k = -2 o_k (q_k - v) / e_k = (o_k / 6) (6 q_k - 6 v) (-2 / e_k)
    const double ck = oc[k] * (a.q[k] - v6) * m2ie[k];
    tb[k] = t2[k] * ck;
    sb[k] = s613[k] * ck;
  }
  gr[0] = 2.0 * oc[0] + tb[0] + sb[0];
  gr[1] = -7.0 * oc[0] - oc[1] - 2.0 * tb[0] - 4.0 * sb[0] + tb[1] + sb[1];
  gr[2] = 11.0 * oc[0] + 5.0 * oc[1] + 2.0 * oc[2] + tb[0] + 3.0 * sb[0] - 2.0 * tb[1] + tb[2] + 3.0 * sb[2];
  gr[3] = 2.0 * oc[1] + 5.0 * oc[2] + tb[1] - sb[1] - 2.0 * tb[2] - 4.0 * sb[2];
  gr[4] = -oc[2] + tb[2] + sb[2];
  return v6 * c6;
}

__device__ __forceinline__ void weno5_cell_value_grad(const double u[5], double eps13, double& vm, double gm[5],
                                                      double& vp, double gp[5]) {
  Weno5VG A, B;
  weno5_vg_parts(u, eps13, A);
  B.q[0] = fma(2.0, u[4], fma(-7.0, u[3], 11.0 * u[2]));
  B.q[1] = fma(2.0, u[1], fma(5.0, u[2], -u[3]));
  B.q[2] = fma(5.0, u[1], fma(2.0, u[2], -u[0]));
  B.w[0] = A.p[2] * A.p[2];
  B.w[1] = A.w[1];
  B.w[2] = 3.0 * A.w[0];
  B.ws = B.w[0] + B.w[1] + B.w[2];
  const double ab = A.ws * B.ws;
  const double Z = rcp_nr(ab * A.ee);
  const double eZ = A.ee * Z;
  const double m2iee = -2.0 * (ab * Z);  // -2 / (e0 e1 e2)
  // shared factors in the plus state's order and mirrored for the minus state
  double t2A[3], sA[3], mA[3], t2B[3], sB[3], mB[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    t2A[k] = 2.0 * A.t[k];
    sA[k] = (6.0 / 13.0) * A.s[k];
    mA[k] = A.p[k] * m2iee;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    t2B[k] = t2A[2 - k];
    sB[k] = sA[2 - k];
    mB[k] = mA[2 - k];
  }
  sB[1] = -sA[1];
  double gr[5];
  vp = weno5_state_grad(A, t2A, sA, mA, B.ws * eZ, gp);
  vm = weno5_state_grad(B, t2B, sB, mB, A.ws * eZ, gr);
#pragma unroll
  for (int k = 0; k < 5; ++k) gm[k] = gr[4 - k];  // derivatives w.r.t. the mirrored stencil's u_{4-k}
}

// minmod face value um1 + minmod(um1 - um2, u0 - um1) / 2 with its adjoint.
__device__ __forceinline__ double minmod_left_adj(double um2, double um1, double u0, double vbar, double ub[3]) {
  const double a = um1 - um2, b = u0 - um1;
  double v = um1;
  ub[1] += vbar;
  if (a * b > 0.0) {
    if (fabs(a) <= fabs(b)) { v += 0.5 * a; ub[1] += 0.5 * vbar; ub[0] -= 0.5 * vbar; }
    else { v += 0.5 * b; ub[2] += 0.5 * vbar; ub[1] -= 0.5 * vbar; }
  }
  return v;
}

// ------------------------------------------------------------- side adjoint
// Recompute one face state (see side_state) and propagate the adjoints of
// its outputs (U, F, lm, lp) to the primitives and Gamma.
// ia = 1 / alpha of the face.  The speeds are those of side_state:
// lambda_pm = alpha (c0 pm sq) / dsp - beta^d with Na = Gamma P + b^2,
// dsp = hs - v^2 Na, hmn = hs - Na, Q = max(gamma^dd dsp - vd^2 hmn, 0),
// sq = sqrt(Na (1 - v^2) Q), c0 = vd hmn.
template <bool CURVED, int DIR>
__device__ __forceinline__ void side_state_adj(const double pr[8], const Geom<double>& m, double gamma, double gfac,
                                               double dgfac, double ia, const double Ub[8], const double Fb[8],
                                               double lmb, double lpb, double prb[8], double& gammab) {
  const double rho = pr[0], P = pr[4];
  const double v[3] = {pr[1], pr[2], pr[3]};
  const double B[3] = {pr[5], pr[6], pr[7]};
  double vl[3], Bl[3];
  if (CURVED) { lower(m.g, v, vl); lower(m.g, B, Bl); }
  else {
#pragma unroll
    for (int i = 0; i < 3; ++i) { vl[i] = v[i]; Bl[i] = B[i]; }
  }
  const double v2 = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
  const double Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const double B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const double omv2 = 1.0 - v2;
  const double W = rsqrt(omv2);
  const double iW = omv2 * W;
  const double ab0 = W * Bv;
  const double b2 = B2 * omv2 + Bv * Bv;
  double bl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) bl[i] = Bl[i] * iW + ab0 * vl[i];
  const double rhoh = rho + gfac * P;
  const double hs = rhoh + b2;
  const double Ps = P + 0.5 * b2;
  const double sg = CURVED ? m.sqrtg : 1.0;
  const double hW2 = hs * W * W;
  const double D = sg * rho * W;
  double S[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) S[i] = sg * (hW2 * vl[i] - ab0 * bl[i]);
  const double tau = sg * (hW2 - Ps - ab0 * ab0) - D;
  double Bc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Bc[i] = sg * B[i];
  const double alpha = CURVED ? m.alpha : 1.0;
  double vt[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) vt[i] = CURVED ? v[i] - m.beta[i] * ia : v[i];
  const double vtd = vt[DIR];
  const double BdiW = Bc[DIR] * iW;
  const double gdd = CURVED ? m.gup_dd : 1.0;
  const double Na = gamma * P + b2;
  const double dsp = hs - v2 * Na;
  const double hmn = hs - Na;
  const double vd = v[DIR];
  const double Q0 = gdd * dsp - vd * vd * hmn;
  // (the clamp, the tests, the square root and the reciprocal as in side_state: fpbits.cuh)
  const double Q = dmax0i(Q0);
  const double sq = sqrt_nr(Na * omv2 * Q);
  const double c0 = vd * hmn;
  const bool sqpos = dgt0i(sq);
  // 1/dsp and 1/sq from one division
  const double sqs = sqpos ? sq : 1.0;
  const double Y = rcp_nr(dsp * sqs);
  const double idsp = sqs * Y, isq = dsp * Y;
  const double id = alpha * idsp;

  // ---- reverse ----
  double rhob = 0, Pb = 0, vb[3] = {0, 0, 0}, Bb[3] = {0, 0, 0};
  double vlb[3] = {0, 0, 0}, Blb[3] = {0, 0, 0}, blb[3] = {0, 0, 0};
  double v2b = 0, Bvb = 0, B2b = 0, omv2b = 0, iWb = 0, Wb = 0, ab0b = 0, b2b = 0;
  double rhohb = 0, hsb = 0, Psb = 0, hW2b = 0, Db = 0, Sb[3], taub = 0, Bcb[3], vtb[3] = {0, 0, 0};
  double gfacb = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) { Sb[i] = Ub[1 + i]; Bcb[i] = Ub[5 + i]; }
  Db = Ub[0];
  taub = Ub[4];
  // speeds
  {
    const double idb = lpb * (c0 + sq) + lmb * (c0 - sq);
    const double c0b = id * (lpb + lmb);
    const double sqb = id * (lpb - lmb);
    double dspb = -id * idsp * idb;
    double Nab = 0, hmnb = 0, vdb = 0;
    if (sqpos) {
      const double Xb = 0.5 * sqb * isq;
      Nab += omv2 * Q * Xb;
      omv2b += Na * Q * Xb;
      const double Qb = Na * omv2 * Xb;
      if (dgt0i(Q0)) {
        dspb += gdd * Qb;
        vdb -= 2.0 * vd * hmn * Qb;
        hmnb -= vd * vd * Qb;
      }
    }
    vdb += hmn * c0b;
    hmnb += vd * c0b;
    hsb += hmnb + dspb;
    Nab -= hmnb + v2 * dspb;
    v2b -= Na * dspb;
    gammab += P * Nab;
    Pb += gamma * Nab;
    b2b += Nab;
    vb[DIR] += vdb;
  }
  // fluxes
  {
    double BdiWb = 0;
    Db += alpha * vtd * Fb[0];
    vtb[DIR] += alpha * D * Fb[0];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double f = alpha * Fb[1 + j];
      Sb[j] += vtd * f;
      vtb[DIR] += S[j] * f;
      if (j == DIR) Psb += sg * f;
      blb[j] -= BdiW * f;
      BdiWb -= bl[j] * f;
    }
    {
      const double f = alpha * Fb[4];
      taub += vtd * f;
      vtb[DIR] += tau * f;
      Psb += sg * v[DIR] * f;
      vb[DIR] += sg * Ps * f;
      ab0b -= BdiW * f;
      BdiWb -= ab0 * f;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k == DIR) continue;
      const double f = alpha * Fb[5 + k];
      Bcb[k] += vtd * f;
      vtb[DIR] += Bc[k] * f;
      Bcb[DIR] -= vt[k] * f;
      vtb[k] -= Bc[DIR] * f;
    }
    Bcb[DIR] += iW * BdiWb;
    iWb += Bc[DIR] * BdiWb;
#pragma unroll
    for (int i = 0; i < 3; ++i) vb[i] += vtb[i];
  }
  // conserved variables
#pragma unroll
  for (int i = 0; i < 3; ++i) Bb[i] += sg * Bcb[i];
  hW2b += sg * taub;
  Psb -= sg * taub;
  ab0b -= 2.0 * sg * ab0 * taub;
  Db -= taub;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    hW2b += sg * vl[i] * Sb[i];
    vlb[i] += sg * hW2 * Sb[i];
    ab0b -= sg * bl[i] * Sb[i];
    blb[i] -= sg * ab0 * Sb[i];
  }
  rhob += sg * W * Db;
  Wb += sg * rho * Db;
  hsb += W * W * hW2b;
  Wb += 2.0 * hs * W * hW2b;
  Pb += Psb;
  b2b += 0.5 * Psb;
  rhohb += hsb;
  b2b += hsb;
  rhob += rhohb;
  Pb += gfac * rhohb;
  gfacb += P * rhohb;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Blb[i] += iW * blb[i];
    iWb += Bl[i] * blb[i];
    ab0b += vl[i] * blb[i];
    vlb[i] += ab0 * blb[i];
  }
  B2b += omv2 * b2b;
  omv2b += B2 * b2b;
  Bvb += 2.0 * Bv * b2b;
  Wb += Bv * ab0b;
  Bvb += W * ab0b;
  iWb -= W * W * Wb;
  omv2b += iWb * 0.5 * W;
  v2b -= omv2b;
  // v2 = v.Gv, Bv = B.Gv, B2 = B.GB; vl = Gv, Bl = GB (G symmetric)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    vb[i] += 2.0 * vl[i] * v2b + Bl[i] * Bvb;
    Bb[i] += vl[i] * Bvb + 2.0 * Bl[i] * B2b;
  }
  double Gvlb[3], GBlb[3];
  if (CURVED) { lower(m.g, vlb, Gvlb); lower(m.g, Blb, GBlb); }
  else {
#pragma unroll
    for (int i = 0; i < 3; ++i) { Gvlb[i] = vlb[i]; GBlb[i] = Blb[i]; }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) { vb[i] += Gvlb[i]; Bb[i] += GBlb[i]; }
  gammab += gfacb * dgfac;  // dgfac = d gfac / d Gamma = -1 / (Gamma - 1)^2
  prb[0] += rhob;
  prb[1] += vb[0];
  prb[2] += vb[1];
  prb[3] += vb[2];
  prb[4] += Pb;
  prb[5] += Bb[0];
  prb[6] += Bb[1];
  prb[7] += Bb[2];
}

// ---------------------------------------------------------------- face adjoint
// Cell-state buffer of one direction (BUF): Wb[((2 q + s) 6 + j) ncell + cell],
// s = 0 the minus state (value at the cell's lower face), 1 the plus state,
// j = 0 the value and 1..5 its derivatives with respect to u_{i-2 .. i+2}.
constexpr int kAdjStateComps = 96;
__device__ __forceinline__ long long adj_state_index(int q, int side, int j, long long ncell, long long cell) {
  return (long long)((2 * q + side) * 6 + j) * ncell + cell;
}

template <int RECON, bool CURVED, int DIR, bool BUF = false>
__device__ __forceinline__ void face_adjoint(const DevGrid& g, const DevParams& p, const double* __restrict__ prim,
                                             const double* __restrict__ metric, long long c, const double Fb[8],
                                             double* __restrict__ prim_bar, double& gammab, double* gsm,
                                             const double* __restrict__ Wb = nullptr) {
  const long long stride = (DIR == 0) ? 1 : ((DIR == 1) ? g.sy : g.sz);
  // primal reconstruction; for WENO5 the five partial derivatives of every
  // face value are kept in shared memory (gsm[j * blockDim.x + tid],
  // j = (2 q + side) * 5 + k) for the reverse sweep below, or (BUF) read
  // from the cell-state buffer: the left state is the plus state of the cell
  // below, the right state the minus state of the cell above
  double pL[8], pR[8];
  const double eps = p.weno_eps;
  if constexpr (BUF) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      pL[q] = __ldg(Wb + adj_state_index(q, 1, 0, g.ncell, c - stride));
      pR[q] = __ldg(Wb + adj_state_index(q, 0, 0, g.ncell, c));
    }
  } else if (RECON == GRMHD_WENO5) {
    const double eps13 = eps * (12.0 / 13.0);
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      double u[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) u[k] = __ldg(prim + q * g.ncell + c + (k - 3) * stride);
      double grL[5], grR[5];
      const double uL[5] = {u[0], u[1], u[2], u[3], u[4]};
      const double uR[5] = {u[5], u[4], u[3], u[2], u[1]};
      weno5_value_grad2(uL, uR, eps13, pL[q], grL, pR[q], grR);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        gsm[((2 * q) * 5 + k) * blockDim.x + threadIdx.x] = grL[k];
        gsm[((2 * q + 1) * 5 + k) * blockDim.x + threadIdx.x] = grR[k];
      }
    }
  } else {
    reconstruct_face<double, RECON>(prim, g.ncell, c, stride, eps, pL, pR);
  }
  Geom<double> m;
  if (CURVED) face_geom<double, DIR>(metric, g.ncell, c, stride, m);
  const bool fbL = !physical_state<double, CURVED>(pL, m);
  const bool fbR = !physical_state<double, CURVED>(pR, m);
  if (fbL)
#pragma unroll
    for (int q = 0; q < 8; ++q) pL[q] = __ldg(prim + q * g.ncell + c - stride);
  if (fbR)
#pragma unroll
    for (int q = 0; q < 8; ++q) pR[q] = __ldg(prim + q * g.ncell + c);
  Side<double> L, R;
  const double ia = CURVED ? 1.0 / m.alpha : 1.0;
  side_state<double, CURVED, DIR, true>(pL, m, p.gamma, p.gfac, L, ia);
  side_state<double, CURVED, DIR, true>(pR, m, p.gamma, p.gfac, R, ia);
  finish_speeds<double, CURVED, DIR>(m, L, R);
  // HLLE reverse
  double FLb[8], FRb[8], ULb[8], URb[8], lmLb = 0, lpLb = 0, lmRb = 0, lpRb = 0;
  // (the bounds, the tests and the reciprocal on the integer pipe / as Newton steps: fpbits.cuh)
  const double xm = dmin0_2i(L.lm, R.lm);
  const double xp = dmax0_2i(L.lp, R.lp);
  const double dd = xp - xm;
  if (dltposi(dd, 1e-300)) {
#pragma unroll
    for (int q = 0; q < 8; ++q) { FLb[q] = FRb[q] = 0.5 * Fb[q]; ULb[q] = URb[q] = 0.0; }
  } else {
    const double inv = rcp_nr(dd);
    double xpb = 0, xmb = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double dU = R.U[q] - L.U[q];
      const double F = (xp * L.F[q] - xm * R.F[q] + xp * xm * dU) * inv;
      FLb[q] = xp * inv * Fb[q];
      FRb[q] = -xm * inv * Fb[q];
      URb[q] = xp * xm * inv * Fb[q];
      ULb[q] = -URb[q];
      xpb += Fb[q] * (L.F[q] + xm * dU - F) * inv;
      xmb += Fb[q] * (-R.F[q] + xp * dU + F) * inv;
    }
    // route through max / min (ties go to the first candidate in the forward order)
    if (dgt0i(xp)) { if (L.lp >= R.lp) lpLb += xpb; else lpRb += xpb; }
    if (!dge0i(xm)) { if (L.lm <= R.lm) lmLb += xmb; else lmRb += xmb; }
  }
  double pLb[8] = {0, 0, 0, 0, 0, 0, 0, 0}, pRb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const double dgfac = -1.0 / ((p.gamma - 1.0) * (p.gamma - 1.0));
  side_state_adj<CURVED, DIR>(pL, m, p.gamma, p.gfac, dgfac, ia, ULb, FLb, lmLb, lpLb, pLb, gammab);
  side_state_adj<CURVED, DIR>(pR, m, p.gamma, p.gfac, dgfac, ia, URb, FRb, lmRb, lpRb, pRb, gammab);
  // reconstruction reverse (stencil values reloaded), scatter to the stencil
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    double ub[6] = {0, 0, 0, 0, 0, 0};
    if (fbL) ub[2] += pLb[q];
    if (fbR) ub[3] += pRb[q];
    if constexpr (BUF) {
      // plus state of the cell below: u_{c-3 .. c+1}; minus state of the cell above: u_{c-2 .. c+2}
      if (!fbL) {
#pragma unroll
        for (int k = 0; k < 5; ++k) ub[k] += __ldg(Wb + adj_state_index(q, 1, 1 + k, g.ncell, c - stride)) * pLb[q];
      }
      if (!fbR) {
#pragma unroll
        for (int k = 0; k < 5; ++k) ub[k + 1] += __ldg(Wb + adj_state_index(q, 0, 1 + k, g.ncell, c)) * pRb[q];
      }
    } else if (RECON == GRMHD_WENO5) {
      if (!fbL) {
#pragma unroll
        for (int k = 0; k < 5; ++k) ub[k] += gsm[((2 * q) * 5 + k) * blockDim.x + threadIdx.x] * pLb[q];
      }
      if (!fbR) {
#pragma unroll
        for (int k = 0; k < 5; ++k) ub[5 - k] += gsm[((2 * q + 1) * 5 + k) * blockDim.x + threadIdx.x] * pRb[q];
      }
    } else {
      double u[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) u[k] = __ldg(prim + q * g.ncell + c + (k - 3) * stride);
      if (!fbL) {
        double t[3] = {0, 0, 0};
        minmod_left_adj(u[1], u[2], u[3], pLb[q], t);
        ub[1] += t[0]; ub[2] += t[1]; ub[3] += t[2];
      }
      if (!fbR) {
        // u0 - minmod(u0 - um1, up1 - u0)/2 is the mirror of the left formula
        double t[3] = {0, 0, 0};
        minmod_left_adj(u[4], u[3], u[2], pRb[q], t);
        ub[4] += t[0]; ub[3] += t[1]; ub[2] += t[2];
      }
    }
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (ub[s] != 0.0) atomicAdd(prim_bar + q * g.ncell + c + (s - 3) * stride, ub[s]);
  }
}

// One thread per face: F_bar = scale * (Lbar_c - Lbar_{c-1}) / dx_d, with
// Lbar = 0 outside the interior.
template <int RECON, bool CURVED>
__global__ void __launch_bounds__(128) rhs_face_adjoint_kernel(DevGrid g, DevParams p, const double* __restrict__ prim,
                                                              const double* __restrict__ metric,
                                                              const double* __restrict__ rhs_bar, double scale,
                                                              double* __restrict__ prim_bar,
                                                              double* __restrict__ gamma_bar, int dsel, int r0,
                                                              int rstep) {
  // dsel < 0: the faces of all three directions; else the dsel-faces at r0,
  // r0 + rstep, ... along dsel (as rhs_face_adjoint_buf_kernel)
  long long nfx = (long long)(g.n[0] + 1) * g.n[1] * g.n[2];
  long long nfy = (long long)g.n[0] * (g.n[1] + 1) * g.n[2];
  long long nfz = (long long)g.n[0] * g.n[1] * (g.n[2] + 1);
  int nd = 0;
  if (dsel >= 0) {
    nd = g.n[dsel] + 1 > r0 ? (g.n[dsel] + 1 - r0 + rstep - 1) / rstep : 0;
    const long long cross = (long long)g.n[0] * g.n[1] * g.n[2] / g.n[dsel];
    nfx = dsel == 0 ? nd * cross : 0;
    nfy = dsel == 1 ? nd * cross : 0;
    nfz = dsel == 2 ? nd * cross : 0;
  }
  const int ex = dsel == 0 ? nd : g.n[0] + 1, ey = dsel == 1 ? nd : g.n[1] + 1;
  const long long total = nfx + nfy + nfz;
  extern __shared__ __align__(16) unsigned char adj_smem[];
  double* gsm = reinterpret_cast<double*>(adj_smem);  // WENO5 partials, 80 per thread
  double gb = 0.0;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    int dir, xi, yi, zi;
    if (f < nfx) {
      dir = 0;
      xi = (int)(f % ex);
      yi = (int)((f / ex) % g.n[1]);
      zi = (int)(f / ((long long)ex * g.n[1]));
    } else if (f < nfx + nfy) {
      const long long ff = f - nfx;
      dir = 1;
      xi = (int)(ff % g.n[0]);
      yi = (int)((ff / g.n[0]) % ey);
      zi = (int)(ff / ((long long)g.n[0] * ey));
    } else {
      const long long ff = f - nfx - nfy;
      dir = 2;
      xi = (int)(ff % g.n[0]);
      yi = (int)((ff / g.n[0]) % g.n[1]);
      zi = (int)(ff / ((long long)g.n[0] * g.n[1]));
    }
    if (dsel >= 0) {
      if (dir == 0) xi = r0 + rstep * xi;
      else if (dir == 1) yi = r0 + rstep * yi;
      else zi = r0 + rstep * zi;
    }
    const long long c = (long long)(zi + g.ng) * g.sz + (long long)(yi + g.ng) * g.sy + (xi + g.ng);
    const long long stride = dir == 0 ? 1 : (dir == 1 ? g.sy : g.sz);
    const int ic = dir == 0 ? xi : (dir == 1 ? yi : zi);
    const bool has_hi = ic < g.n[dir];   // cell c is interior
    const bool has_lo = ic > 0;          // cell c - stride is interior
    double Fb[8];
    const double w = scale * g.idx[dir];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double hi = has_hi ? rhs_bar[q * g.ncell + c] : 0.0;
      const double lo = has_lo ? rhs_bar[q * g.ncell + c - stride] : 0.0;
      Fb[q] = w * (hi - lo);
    }
    if (dir == 0) face_adjoint<RECON, CURVED, 0>(g, p, prim, metric, c, Fb, prim_bar, gb, gsm);
    else if (dir == 1) face_adjoint<RECON, CURVED, 1>(g, p, prim, metric, c, Fb, prim_bar, gb, gsm);
    else face_adjoint<RECON, CURVED, 2>(g, p, prim, metric, c, Fb, prim_bar, gb, gsm);
  }
  add_gamma(p, gb, gamma_bar);
}

// The cell states of direction DIR with their derivatives, for the buffered
// face adjoint: the cells -1 .. n_DIR of every line along DIR (interior
// across), one item per (variable, cell).  Each cell's two states share their
// smoothness indicators (weno5_cell_value_grad).
template <int DIR>
__global__ void __launch_bounds__(128) adj_cell_states_kernel(DevGrid g, DevParams p, const double* __restrict__ prim,
                                                              double* __restrict__ Wb) {
  const int ex = g.n[0] + 2 * (DIR == 0), ey = g.n[1] + 2 * (DIR == 1), ez = g.n[2] + 2 * (DIR == 2);
  const long long m = (long long)ex * ey * ez;
  const long long stride = DIR == 0 ? 1 : (DIR == 1 ? g.sy : g.sz);
  const double eps13 = p.weno_eps * (12.0 / 13.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 8 * m;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / m);
    const long long l = t - q * m;
    const long long lxy = l / ex;
    const int i = (int)(l - lxy * ex) - (DIR == 0), j = (int)(lxy % ey) - (DIR == 1), k = (int)(lxy / ey) - (DIR == 2);
    const long long c = (long long)(k + g.ng) * g.sz + (long long)(j + g.ng) * g.sy + (i + g.ng);
    double u[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) u[a] = __ldg(prim + q * g.ncell + c + (a - 2) * stride);
    double vm, gm[5], vp, gp[5];
    weno5_cell_value_grad(u, eps13, vm, gm, vp, gp);
    Wb[adj_state_index(q, 0, 0, g.ncell, c)] = vm;
    Wb[adj_state_index(q, 1, 0, g.ncell, c)] = vp;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      Wb[adj_state_index(q, 0, 1 + a, g.ncell, c)] = gm[a];
      Wb[adj_state_index(q, 1, 1 + a, g.ncell, c)] = gp[a];
    }
  }
}

// Face adjoint of the DIR-faces from the cell-state buffer (WENO5).  Each
// face adds into the six cells of its stencil along DIR; the faces r0,
// r0 + 6, ... have disjoint stencils, so with rstep = 6 no cell receives two
// adds in one launch (GRMHD_DETERMINISTIC runs r0 = 0 .. 5 in order).  DET:
// the fixed-order Gamma sum, a separate instantiation so that the default
// kernel carries none of it (its reverse was 0.7% slower with a run-time
// switch).
template <bool CURVED, int DIR, bool DET>
__global__ void __launch_bounds__(128) rhs_face_adjoint_buf_kernel(DevGrid g, DevParams p,
                                                                  const double* __restrict__ prim,
                                                                  const double* __restrict__ metric,
                                                                  const double* __restrict__ rhs_bar, double scale,
                                                                  double* __restrict__ prim_bar,
                                                                  double* __restrict__ gamma_bar,
                                                                  const double* __restrict__ Wb, int r0,
                                                                  int rstep) {
  // the DIR-faces at r0, r0 + rstep, ... along DIR (all of them: 0, 1)
  const int nd = g.n[DIR] + 1 > r0 ? (g.n[DIR] + 1 - r0 + rstep - 1) / rstep : 0;
  const int fx = DIR == 0 ? nd : g.n[0], fy = DIR == 1 ? nd : g.n[1], fz = DIR == 2 ? nd : g.n[2];
  const long long total = (long long)fx * fy * fz;
  const long long stride = DIR == 0 ? 1 : (DIR == 1 ? g.sy : g.sz);
  double gb = 0.0;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    const long long fxy = f / fx;
    int xi = (int)(f - fxy * fx), yi = (int)(fxy % fy), zi = (int)(fxy / fy);
    if (DIR == 0) xi = r0 + rstep * xi;
    else if (DIR == 1) yi = r0 + rstep * yi;
    else zi = r0 + rstep * zi;
    const long long c = (long long)(zi + g.ng) * g.sz + (long long)(yi + g.ng) * g.sy + (xi + g.ng);
    const int ic = DIR == 0 ? xi : (DIR == 1 ? yi : zi);
    const bool has_hi = ic < g.n[DIR];  // cell c is interior
    const bool has_lo = ic > 0;         // cell c - stride is interior
    double Fb[8];
    const double w = scale * g.idx[DIR];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double hi = has_hi ? rhs_bar[q * g.ncell + c] : 0.0;
      const double lo = has_lo ? rhs_bar[q * g.ncell + c - stride] : 0.0;
      Fb[q] = w * (hi - lo);
    }
    face_adjoint<GRMHD_WENO5, CURVED, DIR, true>(g, p, prim, metric, c, Fb, prim_bar, gb, nullptr, Wb);
  }
  if constexpr (DET) block_add_gamma_det(gb, gamma_bar);
  else block_add_gamma(gb, gamma_bar);
}

// ------------------------------------------------------------- source adjoint
// Reverse of the Eq. 13 source of one cell (3+1 form as in source_terms):
// given sbar = d(loss)/d(source), add d(loss)/d(primitives) to pbar[8] and
// d(loss)/d(gfac) to gfbar.  Every source component is linear in T^00, T^0i
// and T^ij with coefficients of the metric alone, so their adjoints come
// first; the reverse then runs through b^mu, W, h* and P* to the primitives.
__device__ __forceinline__ void source_reverse(const DevGrid& g, const double* __restrict__ metric,
                                               const double* __restrict__ kij, long long c, const double pr[8],
                                               double gfac, const double sbar[8], double pbar[8], double& gfbar) {
  double a[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) a[q] = __ldg(metric + q * g.ncell + c);
  const double gxx = a[4], gxy = a[5], gxz = a[6], gyy = a[7], gyz = a[8], gzz = a[9];
  const double cxx = gyy * gzz - gyz * gyz, cxy = gxz * gyz - gxy * gzz, cxz = gxy * gyz - gxz * gyy;
  const double cyy = gxx * gzz - gxz * gxz, cyz = gxy * gxz - gxx * gyz, czz = gxx * gyy - gxy * gxy;
  const double det = gxx * cxx + gxy * cxy + gxz * cxz;
  const double idet = 1.0 / det;
  const double sg = sqrt(det);
  const double gu[6] = {cxx * idet, cxy * idet, cxz * idet, cyy * idet, cyz * idet, czz * idet};
  const double alpha = a[0];
  const double beta[3] = {a[1], a[2], a[3]};
  const double gm[6] = {gxx, gxy, gxz, gyy, gyz, gzz};
  const int I6[6] = {0, 0, 0, 1, 1, 2}, J6[6] = {0, 1, 2, 1, 2, 2};
  const double wsym[6] = {1, 2, 2, 1, 2, 1};
  const double asg = alpha * sg;
  const double ia = 1.0 / alpha, ia2 = ia * ia;
  double betal[3];
  lower(gm, beta, betal);
  // adjoints of T^00, T^0i, T^ij (packed like gamma) from the linear source map
  double T00b = 0.0, T0b[3] = {0.0, 0.0, 0.0}, Tijb[6] = {0, 0, 0, 0, 0, 0};
  {
    double dA0[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const long long st = (j == 0) ? 1 : ((j == 1) ? g.sy : g.sz);
      const double w = g.idx[j] * (1.0 / 12.0);
      double d[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        const double* mm = metric + q * g.ncell + c;
        d[q] = (8.0 * (__ldg(mm + st) - __ldg(mm - st)) - (__ldg(mm + 2 * st) - __ldg(mm - 2 * st))) * w;
      }
      dA0[j] = d[0];
      const double wj = sbar[1 + j] * asg;  // momentum j
      if (wj != 0.0) {
        double bbdg = 0.0;
#pragma unroll
        for (int s2 = 0; s2 < 6; ++s2) {
          const int i = I6[s2], k = J6[s2];
          const double dg = d[4 + s2] * wsym[s2];
          bbdg += beta[i] * beta[k] * dg;
          // 0.5 dg (T0_i beta_k + T0_k beta_i) and 0.5 Tij dg
          T0b[i] += wj * 0.5 * dg * beta[k];
          T0b[k] += wj * 0.5 * dg * beta[i];
          Tijb[s2] += wj * 0.5 * dg;
        }
        T00b += wj * (0.5 * bbdg - alpha * d[0]);
        // T0l_i = T00 betal_i + gamma_im T0_m, weighted by d[1 + i]
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          T00b += wj * d[1 + i] * betal[i];
#pragma unroll
          for (int m2 = 0; m2 < 3; ++m2) T0b[m2] += wj * d[1 + i] * gm[sym_index(i, m2)];
        }
      }
    }
    const double we = sbar[4] * asg;  // energy
    if (we != 0.0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) T0b[i] -= we * dA0[i];
      T00b -= we * (beta[0] * dA0[0] + beta[1] * dA0[1] + beta[2] * dA0[2]);
      if (kij) {
        double K[6];
#pragma unroll
        for (int s2 = 0; s2 < 6; ++s2) K[s2] = __ldg(kij + s2 * g.ncell + c);
        double bK[3];
        lower(K, beta, bK);
        T00b += we * (beta[0] * bK[0] + beta[1] * bK[1] + beta[2] * bK[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) T0b[i] += we * 2.0 * bK[i];
#pragma unroll
        for (int s2 = 0; s2 < 6; ++s2) Tijb[s2] += we * K[s2] * wsym[s2];
      }
    }
  }
  // forward values of the fluid part
  const double rho = pr[0], P = pr[4];
  const double v[3] = {pr[1], pr[2], pr[3]};
  const double B[3] = {pr[5], pr[6], pr[7]};
  double vl[3], Bl[3];
  lower(gm, v, vl);
  lower(gm, B, Bl);
  const double v2 = v[0] * vl[0] + v[1] * vl[1] + v[2] * vl[2];
  const double Bv = B[0] * vl[0] + B[1] * vl[1] + B[2] * vl[2];
  const double B2 = B[0] * Bl[0] + B[1] * Bl[1] + B[2] * Bl[2];
  const double omv2 = 1.0 - v2;
  const double iW = sqrt(omv2);
  const double W = 1.0 / iW;
  const double ab0 = W * Bv;
  const double b2 = B2 * omv2 + Bv * Bv;
  const double hs = rho + gfac * P + b2;
  const double b0 = ab0 * ia;
  double vt[3], bu[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    vt[i] = v[i] - beta[i] * ia;
    bu[i] = B[i] * iW + ab0 * vt[i];
  }
  const double hW2 = hs * W * W;
  // reverse through T^00, T^0i, T^ij
  double hW2b = T00b * ia2, Psb = -T00b * ia2, b0b = -2.0 * b0 * T00b;
  double vtb[3] = {0.0, 0.0, 0.0}, bub[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    hW2b += T0b[i] * vt[i] * ia;
    vtb[i] += T0b[i] * hW2 * ia;
    Psb += T0b[i] * beta[i] * ia2;
    b0b -= T0b[i] * bu[i];
    bub[i] -= T0b[i] * b0;
  }
#pragma unroll
  for (int s2 = 0; s2 < 6; ++s2) {
    const int i = I6[s2], j = J6[s2];
    const double t = Tijb[s2];
    hW2b += t * vt[i] * vt[j];
    vtb[i] += t * hW2 * vt[j];
    vtb[j] += t * hW2 * vt[i];
    Psb += t * (gu[s2] - beta[i] * beta[j] * ia2);
    bub[i] -= t * bu[j];
    bub[j] -= t * bu[i];
  }
  // hW2 = hs W^2
  double hsb = hW2b * W * W;
  double Wb = hW2b * 2.0 * hs * W;
  // bu_i = B_i iW + ab0 vt_i ;  b0 = ab0 ia
  double Bb[3], iWb = 0.0, ab0b = b0b * ia;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Bb[i] = bub[i] * iW;
    iWb += bub[i] * B[i];
    ab0b += bub[i] * vt[i];
    vtb[i] += bub[i] * ab0;
  }
  // hs = rho + gfac P + b2 ;  Ps = P + b2 / 2
  const double rhob = hsb;
  double Pb = hsb * gfac + Psb;
  gfbar += hsb * P;
  const double b2b = hsb + 0.5 * Psb;
  // ab0 = W Bv ;  b2 = B2 omv2 + Bv^2
  Wb += ab0b * Bv;
  const double Bvb = ab0b * W + 2.0 * Bv * b2b;
  const double B2b = b2b * omv2;
  double omv2b = b2b * B2;
  // W = 1 / iW ;  iW = sqrt(omv2) ;  omv2 = 1 - v2
  iWb -= Wb * W * W;
  omv2b += iWb * 0.5 * W;
  const double v2b = -omv2b;
  // vt_i = v_i - beta_i / alpha ;  v2 = v.Gv ;  Bv = B.Gv ;  B2 = B.GB
  double vb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    vb[i] = vtb[i] + 2.0 * v2b * vl[i] + Bvb * Bl[i];
    Bb[i] += Bvb * vl[i] + 2.0 * B2b * Bl[i];
  }
  pbar[0] += rhob;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    pbar[1 + i] += vb[i];
    pbar[5 + i] += Bb[i];
  }
  pbar[4] += Pb;
}

__global__ void source_adjoint_kernel(DevGrid g, DevParams p, const double* __restrict__ prim,
                                      const double* __restrict__ metric, const double* __restrict__ kij,
                                      const double* __restrict__ rhs_bar, double scale, double* __restrict__ prim_bar,
                                      double* __restrict__ gamma_bar) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  double gb = 0.0;
  // d gfac / d Gamma for gfac = Gamma / (Gamma - 1)
  const double dgfac = -1.0 / ((p.gamma - 1.0) * (p.gamma - 1.0));
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, t);
    double pr[8], sbar[8], pb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      pr[q] = __ldg(prim + q * g.ncell + c);
      sbar[q] = scale * rhs_bar[q * g.ncell + c];
    }
    double gfb = 0.0;
    source_reverse(g, metric, kij, c, pr, p.gfac, sbar, pb, gfb);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (pb[q] != 0.0) atomicAdd(prim_bar + q * g.ncell + c, pb[q]);
    gb += gfb * dgfac;
  }
  add_gamma(p, gb, gamma_bar);
}

// --------------------------------------------------------- elementwise pieces
// y = a * x + b * y on the interior of nvar fields (x may be NULL: y = b y).
__global__ void axpby_interior_kernel(DevGrid g, int nvar, double a, const double* __restrict__ x, double b,
                                      double* __restrict__ y) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint * nvar;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / nint);
    const long long c = interior_cell(g, t % nint) + q * g.ncell;
    y[c] = (x ? a * x[c] : 0.0) + (b != 0.0 ? b * y[c] : 0.0);
  }
}

// L += sum_interior rho^2 sqrt(gamma) dV ;  prim_bar[rho] += 2 rho sqrt(gamma) dV * lbar
__global__ void density_l2_kernel(DevGrid g, const double* __restrict__ prim, const double* __restrict__ metric,
                                  double lbar, double* __restrict__ loss, double* __restrict__ prim_bar) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  const double dV = g.dx[0] * g.dx[1] * g.dx[2];
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nint;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, t);
    CellMetric m;
    cell_metric(metric, g.ncell, c, m);
    const double rho = prim[c];
    acc += rho * rho * m.sqrtg * dV;
    if (prim_bar) prim_bar[c] += 2.0 * rho * m.sqrtg * dV * lbar;
  }
  if (loss) block_add_gamma(acc, loss);
}

int blocks_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)(b < 1 ? 1 : b);
}

template <bool CURVED, int DIR>
cudaError_t launch_face_adjoint_dir(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                                    const double* rhs_bar, double scale, double* prim_bar, double* gamma_bar,
                                    double* Wb, cudaStream_t s) {
  const long long cells = 8LL * (g.n[0] + 2 * (DIR == 0)) * (g.n[1] + 2 * (DIR == 1)) * (g.n[2] + 2 * (DIR == 2));
  adj_cell_states_kernel<DIR><<<blocks_for(cells, 128), 128, 0, s>>>(g, p, prim, Wb);
  const long long faces = (long long)(g.n[0] + (DIR == 0)) * (g.n[1] + (DIR == 1)) * (g.n[2] + (DIR == 2));
  if (p.flags & GRMHD_DETERMINISTIC) {
    // six launches, the faces of one residue of their index mod 6 each
    for (int r = 0; r < 6; ++r)
      rhs_face_adjoint_buf_kernel<CURVED, DIR, true><<<blocks_for(faces / 6 + 1, 128), 128, 0, s>>>(
          g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, Wb, r, 6);
  } else {
    rhs_face_adjoint_buf_kernel<CURVED, DIR, false><<<blocks_for(faces, 128), 128, 0, s>>>(
        g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, Wb, 0, 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_rhs_adjoint(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                               const double* kij, const double* rhs_bar, double scale, double* prim_bar,
                               double* gamma_bar, cudaStream_t s, double* Wb = nullptr) {
  if (Wb && p.recon == GRMHD_WENO5) {
    // WENO5 with a cell-state buffer: per direction, the cell states with
    // their derivatives, then the faces
    cudaError_t e;
    if (metric) {
      if ((e = launch_face_adjoint_dir<true, 0>(g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, Wb, s)) ||
          (e = launch_face_adjoint_dir<true, 1>(g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, Wb, s)) ||
          (e = launch_face_adjoint_dir<true, 2>(g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, Wb, s)))
        return e;
    } else {
      if ((e = launch_face_adjoint_dir<false, 0>(g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, Wb, s)) ||
          (e = launch_face_adjoint_dir<false, 1>(g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, Wb, s)) ||
          (e = launch_face_adjoint_dir<false, 2>(g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, Wb, s)))
        return e;
      return cudaSuccess;
    }
    const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
    source_adjoint_kernel<<<blocks_for(nint, 128), 128, 0, s>>>(g, p, prim, metric, kij, rhs_bar, scale, prim_bar,
                                                                gamma_bar);
    return cudaGetLastError();
  }
  const long long faces = (long long)(g.n[0] + 1) * g.n[1] * g.n[2] + (long long)g.n[0] * (g.n[1] + 1) * g.n[2] +
                          (long long)g.n[0] * g.n[1] * (g.n[2] + 1);
  const int nb = blocks_for(faces, 128);
  const bool weno = p.recon == GRMHD_WENO5;
  const size_t smem = weno ? (size_t)80 * 128 * sizeof(double) : 0;
  void (*k)(DevGrid, DevParams, const double*, const double*, const double*, double, double*, double*, int, int, int);
  if (metric) k = weno ? rhs_face_adjoint_kernel<GRMHD_WENO5, true> : rhs_face_adjoint_kernel<GRMHD_MINMOD, true>;
  else k = weno ? rhs_face_adjoint_kernel<GRMHD_WENO5, false> : rhs_face_adjoint_kernel<GRMHD_MINMOD, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.flags & GRMHD_DETERMINISTIC) {
    // per direction, six launches by face index mod 6 (disjoint stencils)
    for (int d = 0; d < 3; ++d)
      for (int r = 0; r < 6; ++r)
        k<<<blocks_for(faces / 18 + 1, 128), 128, smem, s>>>(g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar,
                                                             d, r, 6);
  } else {
    k<<<nb, 128, smem, s>>>(g, p, prim, metric, rhs_bar, scale, prim_bar, gamma_bar, -1, 0, 1);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || !metric) return e;
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  source_adjoint_kernel<<<blocks_for(nint, 128), 128, 0, s>>>(g, p, prim, metric, kij, rhs_bar, scale, prim_bar,
                                                              gamma_bar);
  return cudaGetLastError();
}

}  // namespace grmhd

using namespace grmhd;

namespace {

bool al8(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 7u) == 0; }
size_t r256(size_t b) { return (b + 255) & ~(size_t)255; }

int check_common(const grmhd_grid* grid, const grmhd_params* params, const double* metric) {
  if (!grid || !params) return GRMHD_ERR_ARG;
  if (params->precision != GRMHD_FP64) return GRMHD_ERR_ARG;  // the adjoint is of the FP64 method
  if ((params->flags & ~(GRMHD_REUSE_GEOMETRY | GRMHD_NEWMAN_HAMLIN | GRMHD_SINGLE_PASS | GRMHD_DETERMINISTIC)) != 0)
    return GRMHD_ERR_ARG;
  if (params->eos != GRMHD_EOS_IDEAL) return GRMHD_ERR_ARG;    // ... with the Gamma-law
  if (!(params->gamma > 1.0 && params->gamma <= 3.0)) return GRMHD_ERR_ARG;
  if (params->recon != GRMHD_WENO5 && params->recon != GRMHD_MINMOD) return GRMHD_ERR_ARG;
  if (params->bc != GRMHD_BC_PERIODIC && params->bc != GRMHD_BC_COPY) return GRMHD_ERR_ARG;
  if (params->nr_maxit < 1 || !(params->nr_tol > 0.0) || !(params->weno_eps > 0.0)) return GRMHD_ERR_ARG;
  if (!(params->rho_atm > 0.0) || !(params->p_atm > 0.0) || params->tile < 0 || params->tile > 4) return GRMHD_ERR_ARG;
  const int min_ng = params->recon == GRMHD_WENO5 ? 3 : 2;
  if (grid->ng < min_ng || grid->ng > 16) return GRMHD_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (grid->n[d] < 1 || grid->n[d] > (1 << 20) || !(grid->dx[d] > 0.0)) return GRMHD_ERR_ARG;
  if (metric && !al8(metric)) return GRMHD_ERR_ARG;
  return GRMHD_OK;
}

int st(cudaError_t e) { return e == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA; }

cudaError_t axpby(const DevGrid& g, double a, const double* x, double b, double* y, cudaStream_t s) {
  const long long n = (long long)g.n[0] * g.n[1] * g.n[2] * 8;
  axpby_interior_kernel<<<blocks_for(n, 256), 256, 0, s>>>(g, 8, a, x, b, y);
  return cudaGetLastError();
}

cudaError_t c2p_adjoint(const DevGrid& g, const DevParams& p, const double* prim, const double* metric,
                        const double* prim_bar, double* cons_bar, double* gamma_bar, int32_t* nsing, cudaStream_t s) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  con2prim_adjoint_kernel<<<blocks_for(nint, 128), 128, 0, s>>>(g, p, prim, metric, prim_bar, cons_bar, gamma_bar,
                                                                 nsing);
  return cudaGetLastError();
}

cudaError_t ghost_adjoint(const DevGrid& g, int bc, int nvar, double* f, cudaStream_t s) {
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  fill_ghosts_adjoint_kernel<<<blocks_for(nint, 128), 128, 0, s>>>(g, bc, nvar, f);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int grmhd_rhs_adjoint(const grmhd_grid* grid, const grmhd_params* params, const double* prim, const double* metric,
                      const double* kij, const double* rhs_bar, double* prim_bar, double* gamma_bar, void* stream) {
  int e = check_common(grid, params, metric);
  if (e) return e;
  if (!prim || !rhs_bar || !prim_bar || !gamma_bar || !al8(prim) || !al8(rhs_bar) || !al8(prim_bar) || !al8(gamma_bar))
    return GRMHD_ERR_ARG;
  if (kij && (!metric || !al8(kij))) return GRMHD_ERR_ARG;
  return st(launch_rhs_adjoint(make_grid(*grid), make_params(*params), prim, metric, kij, rhs_bar, 1.0, prim_bar,
                               gamma_bar, (cudaStream_t)stream));
}

int grmhd_con2prim_adjoint(const grmhd_grid* grid, const grmhd_params* params, const double* prim,
                           const double* metric, const double* prim_bar, double* cons_bar, double* gamma_bar,
                           int32_t* nsingular, void* stream) {
  int e = check_common(grid, params, metric);
  if (e) return e;
  if (!prim || !prim_bar || !cons_bar || !gamma_bar || !al8(prim) || !al8(prim_bar) || !al8(cons_bar)) return GRMHD_ERR_ARG;
  return st(c2p_adjoint(make_grid(*grid), make_params(*params), prim, metric, prim_bar, cons_bar, gamma_bar,
                        nsingular, (cudaStream_t)stream));
}

int grmhd_prim2con_adjoint(const grmhd_grid* grid, const grmhd_params* params, const double* prim,
                           const double* metric, const double* cons_bar, double* prim_bar, double* gamma_bar,
                           void* stream) {
  int e = check_common(grid, params, metric);
  if (e) return e;
  if (!prim || !prim_bar || !cons_bar || !gamma_bar || !al8(prim) || !al8(prim_bar) || !al8(cons_bar)) return GRMHD_ERR_ARG;
  const DevGrid g = make_grid(*grid);
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  prim2con_adjoint_kernel<<<blocks_for(nint, 128), 128, 0, (cudaStream_t)stream>>>(g, make_params(*params), prim, metric,
                                                                                     cons_bar, prim_bar, gamma_bar);
  return st(cudaGetLastError());
}

int grmhd_fill_ghosts_adjoint(const grmhd_grid* grid, int32_t bc, int32_t nvar, double* field_bar, void* stream) {
  if (!grid || !field_bar || !al8(field_bar) || nvar < 1 || nvar > 64) return GRMHD_ERR_ARG;
  if (bc != GRMHD_BC_PERIODIC && bc != GRMHD_BC_COPY) return GRMHD_ERR_ARG;
  if (grid->ng < 0 || grid->ng > 16) return GRMHD_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (grid->n[d] < 1 || grid->n[d] > (1 << 20)) return GRMHD_ERR_ARG;
  return st(ghost_adjoint(make_grid(*grid), bc, nvar, field_bar, (cudaStream_t)stream));
}

int grmhd_density_l2(const grmhd_grid* grid, const double* prim, const double* metric, double lbar, double* loss,
                     double* prim_bar, void* stream) {
  if (!grid || !prim || !al8(prim) || (metric && !al8(metric)) || (!loss && !prim_bar)) return GRMHD_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (grid->n[d] < 1 || grid->n[d] > (1 << 20) || !(grid->dx[d] > 0.0)) return GRMHD_ERR_ARG;
  const DevGrid g = make_grid(*grid);
  const long long nint = (long long)g.n[0] * g.n[1] * g.n[2];
  density_l2_kernel<<<blocks_for(nint, 256), 256, 0, (cudaStream_t)stream>>>(g, prim, metric, lbar, loss, prim_bar);
  return st(cudaGetLastError());
}

size_t grmhd_rk_adjoint_workspace_bytes(const grmhd_grid* grid, int32_t scheme) {
  if (!grid || (scheme != GRMHD_RK2 && scheme != GRMHD_RK3)) return 0;
  for (int d = 0; d < 3; ++d)
    if (grid->n[d] < 1 || grid->n[d] > (1 << 20)) return 0;
  const DevGrid g = make_grid(*grid);
  const size_t field = r256((size_t)8 * g.ncell * sizeof(double));
  const int stages = scheme == GRMHD_RK3 ? 3 : 2;
  // + the cell-state buffer of the WENO5 face adjoint (one direction at a time)
  return (size_t)(1 + stages + 1 + 1 + 2) * field + r256((size_t)kAdjStateComps * g.ncell * sizeof(double));
}

int grmhd_rk_step_adjoint(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt,
                          const double* cons, const double* prim, const double* metric, const double* kij,
                          const double* stage_prims, double* cons_bar, double* prim_bar, double* gamma_bar,
                          void* ws, size_t ws_bytes, void* stream) {
  int e = check_common(grid, params, metric);
  if (e) return e;
  if (scheme != GRMHD_RK2 && scheme != GRMHD_RK3) return GRMHD_ERR_ARG;
  if (!(dt > 0.0) || !cons || !prim || !cons_bar || !prim_bar || !gamma_bar || !ws) return GRMHD_ERR_ARG;
  if (!al8(cons) || !al8(prim) || !al8(cons_bar) || !al8(prim_bar) || !al8(gamma_bar)) return GRMHD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return GRMHD_ERR_ARG;
  if (kij && (!metric || !al8(kij))) return GRMHD_ERR_ARG;
  if (ws_bytes < grmhd_rk_adjoint_workspace_bytes(grid, scheme)) return GRMHD_ERR_SIZE;
  const DevGrid g = make_grid(*grid);
  const DevParams p = make_params(*params);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t field = r256((size_t)8 * g.ncell * sizeof(double));
  const size_t nbytes = (size_t)8 * g.ncell * sizeof(double);
  const int ns = scheme == GRMHD_RK3 ? 3 : 2;
  char* base = static_cast<char*>(ws);
  double* W = reinterpret_cast<double*>(base);
  double* Pst[4];
  Pst[0] = const_cast<double*>(prim);
  for (int k = 1; k <= ns; ++k) Pst[k] = reinterpret_cast<double*>(base + (size_t)k * field);
  double* A = reinterpret_cast<double*>(base + (size_t)(ns + 1) * field);
  double* Bacc = reinterpret_cast<double*>(base + (size_t)(ns + 2) * field);
  double* Pn = reinterpret_cast<double*>(base + (size_t)(ns + 3) * field);
  double* Pk = reinterpret_cast<double*>(base + (size_t)(ns + 4) * field);
  double* Wb = reinterpret_cast<double*>(base + (size_t)(ns + 5) * field);
  double c0[3], c1[3], cr[3];
  if (ns == 3) {
    c0[0] = 1.0; c1[0] = 0.0; cr[0] = 1.0;
    c0[1] = 0.75; c1[1] = 0.25; cr[1] = 0.25;
    c0[2] = 1.0 / 3.0; c1[2] = 2.0 / 3.0; cr[2] = 2.0 / 3.0;
  } else {
    c0[0] = 1.0; c1[0] = 0.0; cr[0] = 1.0;
    c0[1] = 0.5; c1[1] = 0.5; cr[1] = 0.5;
  }
  if (stage_prims) {
    if (!al8(stage_prims)) return GRMHD_ERR_ARG;
    for (int k = 1; k <= ns; ++k) Pst[k] = const_cast<double*>(stage_prims) + (size_t)(k - 1) * 8 * g.ncell;
  }
  // recompute the stages exactly as grmhd_rk_step does (unless recorded)
  if (!stage_prims && cudaMemcpyAsync(W, cons, nbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  for (int k = 0; k < ns && !stage_prims; ++k) {
    StageEpilogue ep;
    ep.fb = nullptr;
    ep.faces = nullptr;
    ep.states = nullptr;
    ep.rhs = nullptr;
    ep.u = W;
    ep.u0 = cons;
    ep.acc_in = nullptr;
    ep.acc_out = nullptr;
    ep.c0 = c0[k];
    ep.c1 = c1[k];
    ep.cr = cr[k] * dt;
    ep.ca = ep.wa = ep.wr = 0.0;
    if (launch_rhs_fp64(g, p, Pst[k], metric, kij, ep, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (cudaMemcpyAsync(Pst[k + 1], Pst[k], nbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (launch_con2prim(g, p, W, metric, Pst[k + 1], nullptr, nullptr, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (launch_fill_ghosts(g, p.bc, 8, Pst[k + 1], s) != cudaSuccess) return GRMHD_ERR_CUDA;
  }
  // reverse sweep
  if (cudaMemcpyAsync(A, cons_bar, nbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaMemsetAsync(Bacc, 0, nbytes, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaMemcpyAsync(Pn, prim_bar, nbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  for (int k = ns - 1; k >= 0; --k) {
    if (ghost_adjoint(g, p.bc, 8, Pn, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (c2p_adjoint(g, p, Pst[k + 1], metric, Pn, A, gamma_bar, nullptr, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (axpby(g, c0[k], A, 1.0, Bacc, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (cudaMemsetAsync(Pk, 0, nbytes, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (launch_rhs_adjoint(g, p, Pst[k], metric, kij, A, cr[k] * dt, Pk, gamma_bar, s, Wb) != cudaSuccess)
      return GRMHD_ERR_CUDA;
    if (k >= 1) {
      if (axpby(g, 0.0, nullptr, c1[k], A, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    } else if (c1[0] != 0.0) {
      if (axpby(g, c1[0], A, 1.0, Bacc, s) != cudaSuccess) return GRMHD_ERR_CUDA;
    }
    double* t = Pn;
    Pn = Pk;
    Pk = t;
  }
  if (cudaMemcpyAsync(cons_bar, Bacc, nbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaMemcpyAsync(prim_bar, Pn, nbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GRMHD_ERR_CUDA;
  return GRMHD_OK;
}

}  // extern "C"
