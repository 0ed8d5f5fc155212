// Constrained transport (Sec. 3: the field lives on a staggered grid so that
// its discrete divergence stays zero).  The densitised field sqrt(gamma) B^a
// is held on the lower a-face of every cell; the electric field on the cell
// edges is the mean of the four field fluxes of the faces that meet there,
// and the faces are advanced by its discrete curl, so that the discrete
// divergence of every cell changes by a sum that cancels exactly.
//
// Layouts (array indices, ghosts included, x fastest):
//   b [a * ncell + cell]        field component a on the lower a-face
//   fb[(3 d + a) * ncell + cell] flux of B^a through the lower d-face (a != d;
//                               the entries a == d are not used)
//   E [c * ncell + cell]        edge field on the c-edge through the cell's
//                               corner lower in the other two axes
// Face ranges (interior coordinates): the a-faces have a-index 0 .. n_a and
// interior transverse indices; fb is needed for d-index 0 .. n_d and
// transverse indices -1 .. n (one ring of ghost rows around the block); the
// RHS launch fills it (StageEpilogue::fb: the tiles, then the ring kernel).
#include <cmath>

#include "rhs.cuh"

namespace grmhd {

namespace {

int ct_blocks(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)b;
}

__device__ __forceinline__ long long cell_at(const DevGrid& g, int i, int j, int k) {
  return (long long)(k + g.ng) * g.sz + (long long)(j + g.ng) * g.sy + (i + g.ng);
}

__device__ __forceinline__ long long axis_stride(const DevGrid& g, int d) {
  return d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
}

// Edge fields: E[c * ncell + y] = E_c at the c-edge through the corner of
// cell y that is lower in a and b, (c, a, b) cyclic, for every corner of the
// interior cells and the corners on the upper block faces (interior
// coordinates 0 .. n per axis).  Each edge is formed once: the face update
// reads four of them (FP64 throughput is what bounds this path).
__global__ void ct_edges_kernel(DevGrid g, const double* __restrict__ fb, double* __restrict__ E) {
  const long long ex = g.n[0] + 1, ey = g.n[1] + 1, total = ex * ey * (g.n[2] + 1);
  const long long n = g.ncell;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long q = t / ex;
    const long long y = cell_at(g, (int)(t - q * ex), (int)(q % ey), (int)(q / ey));
    // E_0 (a = 1, b = 2), E_1 (a = 2, b = 0), E_2 (a = 0, b = 1)
    E[y] = 0.25 * ((fb[(3 * 2 + 1) * n + y - g.sy] + fb[(3 * 2 + 1) * n + y]) -
                   (fb[(3 * 1 + 2) * n + y - g.sz] + fb[(3 * 1 + 2) * n + y]));
    E[n + y] = 0.25 * ((fb[(3 * 0 + 2) * n + y - g.sz] + fb[(3 * 0 + 2) * n + y]) -
                       (fb[(3 * 2 + 0) * n + y - 1] + fb[(3 * 2 + 0) * n + y]));
    E[2 * n + y] = 0.25 * ((fb[(3 * 1 + 0) * n + y - 1] + fb[(3 * 1 + 0) * n + y]) -
                           (fb[(3 * 0 + 1) * n + y - g.sy] + fb[(3 * 0 + 1) * n + y]));
  }
}

// Rate of the lower A-face of cell x: -(E_C[+e_B] - E_C)/dx_B + (E_B[+e_C] - E_B)/dx_C, (A, B, C) cyclic.
template <int A>
__device__ __forceinline__ double face_rate(const DevGrid& g, const double* __restrict__ E, long long x) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  const double* Ec = E + C * g.ncell;
  const double* Eb = E + B * g.ncell;
  return (Eb[x + axis_stride(g, C)] - Eb[x]) * g.idx[C] - (Ec[x + axis_stride(g, B)] - Ec[x]) * g.idx[B];
}

// Every face of the face ranges: its rate (into rate, if set), and, with b
// set, the stage update b <- c0 b0 + c1 b + cr rate (+ ca acc_in),
// acc_out <- wa acc_in + wr rate (acc_in and acc_out may be one buffer).
__global__ void ct_faces_kernel(DevGrid g, const double* __restrict__ E, double* __restrict__ rate,
                                double* __restrict__ bf, const double* __restrict__ b0,
                                const double* acc_in, double* acc_out, double c0,
                                double c1, double cr, double ca, double wa, double wr) {
  const long long nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long f0 = (nx + 1) * ny * nz, f1 = nx * (ny + 1) * nz, total = f0 + f1 + nx * ny * (nz + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = t < f0 ? 0 : (t < f0 + f1 ? 1 : 2);
    const long long r = t - (a == 0 ? 0 : (a == 1 ? f0 : f0 + f1));
    const long long ex = nx + (a == 0), ey = ny + (a == 1);
    const long long q = r / ex;
    const int i = (int)(r - q * ex), j = (int)(q % ey), k = (int)(q / ey);
    const long long x = cell_at(g, i, j, k);
    const double L = a == 0 ? face_rate<0>(g, E, x) : (a == 1 ? face_rate<1>(g, E, x) : face_rate<2>(g, E, x));
    const long long o = a * g.ncell + x;
    if (rate) rate[o] = L;
    if (bf) {
      const double ain = acc_in ? acc_in[o] : 0.0;
      bf[o] = c0 * b0[o] + c1 * bf[o] + cr * L + ca * ain;
      if (acc_out) acc_out[o] = wa * ain + wr * L;
    }
  }
}

// Interior cells: the cell field is the mean of its two faces.
__global__ void ct_face_to_cell_kernel(DevGrid g, const double* __restrict__ bf, double* __restrict__ cons) {
  const long long nx = g.n[0], ny = g.n[1], total = nx * ny * g.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long x = cell_at(g, (int)(t % nx), (int)((t / nx) % ny), (int)(t / (nx * ny)));
#pragma unroll
    for (int a = 0; a < 3; ++a)
      cons[(5 + a) * g.ncell + x] = 0.5 * (bf[a * g.ncell + x] + bf[a * g.ncell + x + axis_stride(g, a)]);
  }
}

// Primitive field of every interior cell from the face field: B^a = (mean of
// the cell's two a-faces) / sqrt(gamma) of the cell (flat: sqrt(gamma) = 1).
__global__ void ct_cell_field_kernel(DevGrid g, const double* __restrict__ bf, const double* __restrict__ metric,
                                     double* __restrict__ prim) {
  const long long nx = g.n[0], ny = g.n[1], total = nx * ny * g.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long x = cell_at(g, (int)(t % nx), (int)((t / nx) % ny), (int)(t / (nx * ny)));
    double isg = 1.0;
    if (metric) {
      const double xx = metric[4 * g.ncell + x], xy = metric[5 * g.ncell + x], xz = metric[6 * g.ncell + x];
      const double yy = metric[7 * g.ncell + x], yz = metric[8 * g.ncell + x], zz = metric[9 * g.ncell + x];
      const double det = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
      isg = 1.0 / sqrt(det);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
      prim[(5 + a) * g.ncell + x] = 0.5 * (bf[a * g.ncell + x] + bf[a * g.ncell + x + axis_stride(g, a)]) * isg;
  }
}

// Discrete divergence of every cell (0 outside the interior); the largest
// |div| into *maxabs (as the bit pattern of a non-negative double, whose
// integer order is its numeric order).
__global__ void ct_divergence_kernel(DevGrid g, const double* __restrict__ bf, double* __restrict__ div,
                                     unsigned long long* __restrict__ maxabs) {
  unsigned long long mx = 0;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < g.ncell;
       x += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(x % g.N[0]) - g.ng, j = (int)((x / g.N[0]) % g.N[1]) - g.ng, k = (int)(x / g.sz) - g.ng;
    double dv = 0.0;
    if (i >= 0 && i < g.n[0] && j >= 0 && j < g.n[1] && k >= 0 && k < g.n[2]) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
        dv = dv + (bf[a * g.ncell + x + axis_stride(g, a)] - bf[a * g.ncell + x]) / g.dx[a];
    }
    if (div) div[x] = dv;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(dv));
    mx = bits > mx ? bits : mx;
  }
  if (maxabs) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_down_sync(0xffffffffu, mx, o);
      mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(maxabs, mx);
  }
}

}  // namespace

cudaError_t launch_ct_faces(const DevGrid& g, const double* fb, double* E, double* rate, double* b, const double* b0,
                            const double* acc_in, double* acc_out, double c0, double c1, double cr, double ca,
                            double wa, double wr, cudaStream_t s) {
  const long long nx = g.n[0], ny = g.n[1], nz = g.n[2];
  ct_edges_kernel<<<ct_blocks((nx + 1) * (ny + 1) * (nz + 1), 256), 256, 0, s>>>(g, fb, E);
  const long long total = (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1);
  ct_faces_kernel<<<ct_blocks(total, 256), 256, 0, s>>>(g, E, rate, b, b0, acc_in, acc_out, c0, c1, cr, ca, wa, wr);
  return cudaGetLastError();
}

cudaError_t launch_ct_face_to_cell(const DevGrid& g, const double* b, double* cons, cudaStream_t s) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  ct_face_to_cell_kernel<<<ct_blocks(total, 256), 256, 0, s>>>(g, b, cons);
  return cudaGetLastError();
}

cudaError_t launch_ct_cell_field(const DevGrid& g, const double* b, const double* metric, double* prim,
                                 cudaStream_t s) {
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  ct_cell_field_kernel<<<ct_blocks(total, 256), 256, 0, s>>>(g, b, metric, prim);
  return cudaGetLastError();
}

cudaError_t launch_ct_divergence(const DevGrid& g, const double* b, double* div, double* maxabs, cudaStream_t s) {
  if (maxabs) {
    const cudaError_t e = cudaMemsetAsync(maxabs, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
  }
  ct_divergence_kernel<<<ct_blocks(g.ncell, 256), 256, 0, s>>>(g, b, div,
                                                               reinterpret_cast<unsigned long long*>(maxabs));
  return cudaGetLastError();
}

}  // namespace grmhd
