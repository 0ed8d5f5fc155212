"""Device check of the paired FP32 side states (csrc/physics.cuh:
side_states_x2, physical_states_x2).

The mixed RHS forms the left and right side states of a face in paired FP32
instructions, one side per lane.  Its operations are those of the scalar
side_state<float, CURVED, 0, true, true> in another rounding order, so it is
compared, like the scalar form, with the FP64 side_state on random physical
states and metrics: conserved vector, flux, speed numerators and speed
denominator, each normwise.  The paired form must be as accurate as the
scalar one (within a factor of two of its largest error, or below 1e-6), and
its physical-state checks must agree with physical_state<float>.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2210_17509_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

CHECK = r"""
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include "physics.cuh"
using namespace grmhd;

__device__ __host__ inline uint64_t mix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ double uni(uint64_t i, int k) { return (double)(mix(i * 64 + k) >> 11) * 0x1p-53; }  // [0, 1)

// a random physical state of cell-centre magnitudes, |v| < 0.9 in the metric g
__device__ void state(uint64_t i, int side, const double g[6], double pr[8]) {
  const int b = 16 * side;
  pr[0] = exp(log(1e-3) * uni(i, b));          // rho in (1e-3, 1]
  pr[4] = exp(log(1e-4) * uni(i, b + 1));      // P in (1e-4, 1]
  double v[3];
  for (int k = 0; k < 3; ++k) v[k] = uni(i, b + 2 + k) - 0.5;
  const double vl0 = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
  const double vl1 = g[1] * v[0] + g[3] * v[1] + g[4] * v[2];
  const double vl2 = g[2] * v[0] + g[4] * v[1] + g[5] * v[2];
  const double v2 = v[0] * vl0 + v[1] * vl1 + v[2] * vl2;
  const double s = v2 > 0.8 ? sqrt(0.8 / v2) : 1.0;
  for (int k = 0; k < 3; ++k) pr[1 + k] = s * v[k];
  for (int k = 0; k < 3; ++k) pr[5 + k] = 2.0 * uni(i, b + 5 + k) - 1.0;
}

template <class A, class B>
__device__ float err(const A* a, const B* ref, int n) {
  double sc = 0.0, e = 0.0;
  for (int k = 0; k < n; ++k) sc = fmax(sc, fabs((double)ref[k]));
  for (int k = 0; k < n; ++k) e = fmax(e, fabs((double)a[k] - (double)ref[k]));
  return sc > 0.0 ? (float)(e / sc) : (float)e;
}

// out[0..3]: paired errors (U, F, speed numerators, denominators); out[4..7]: scalar FP32 errors;
// cnt[0]: check disagreements, cnt[1]: samples with both sides physical
template <bool CURVED>
__global__ void check(long long n, float* out, unsigned long long* cnt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Geom<double> md;
    md.alpha = 0.5 + 0.5 * uni(i, 40);
    for (int k = 0; k < 3; ++k) md.beta[k] = 0.6 * uni(i, 41 + k) - 0.3;
    double d[6];
    for (int k = 0; k < 6; ++k) d[k] = 0.2 * uni(i, 44 + k) - 0.1;
    const double gg[6] = {1.0 + 0.5 * uni(i, 50) + d[0], d[1], d[2], 1.0 + 0.5 * uni(i, 51) + d[3], d[4],
                          1.0 + 0.5 * uni(i, 52) + d[5]};
    for (int k = 0; k < 6; ++k) md.g[k] = CURVED ? gg[k] : (k == 0 || k == 3 || k == 5 ? 1.0 : 0.0);
    if (!CURVED) { md.alpha = 1.0; md.beta[0] = md.beta[1] = md.beta[2] = 0.0; }
    const double cyy = md.g[0] * md.g[5] - md.g[2] * md.g[2], cxx = md.g[3] * md.g[5] - md.g[4] * md.g[4];
    const double det = md.g[0] * cxx - md.g[1] * (md.g[1] * md.g[5] - md.g[4] * md.g[2]) +
                       md.g[2] * (md.g[1] * md.g[4] - md.g[3] * md.g[2]);
    (void)cyy;
    md.gup_dd = cxx / det;
    md.sqrtg = sqrt(det);
    md.ia = 1.0 / md.alpha;
    Geom<float> mf;
    mf.alpha = (float)md.alpha;
    for (int k = 0; k < 3; ++k) mf.beta[k] = (float)md.beta[k];
    for (int k = 0; k < 6; ++k) mf.g[k] = (float)md.g[k];
    mf.gup_dd = (float)md.gup_dd;
    mf.sqrtg = (float)md.sqrtg;
    mf.ia = 1.0f / mf.alpha;
    double pL[8], pR[8];
    state(i, 0, md.g, pL);
    state(i, 1, md.g, pR);
    float fL[8], fR[8];
    for (int q = 0; q < 8; ++q) { fL[q] = (float)pL[q]; fR[q] = (float)pR[q]; }
    // the checks: paired against scalar, on these and on states pushed out of the physical range
    float xL[8], xR[8];
    for (int q = 0; q < 8; ++q) { xL[q] = fL[q]; xR[q] = fR[q]; }
    const int mode = (int)(mix(i * 64 + 60) % 4);
    if (mode == 1) xL[0] = -xL[0];
    if (mode == 2) xR[4] = -0.0f;
    if (mode == 3) { xL[1] *= 3.0f; xR[2] *= 3.0f; }
    bool okL, okR;
    physical_states_x2<CURVED>(xL, xR, mf, okL, okR);
    if (okL != physical_state<float, CURVED>(xL, mf) || okR != physical_state<float, CURVED>(xR, mf))
      atomicAdd(cnt, 1ull);
    const double gam = 5.0 / 3.0, gfac = gam / (gam - 1.0);
    Side<double> dL, dR;
    side_state<double, CURVED, 0, true, true>(pL, md, gam, gfac, dL, md.ia);
    side_state<double, CURVED, 0, true, true>(pR, md, gam, gfac, dR, md.ia);
    Side<float> sL, sR, qL, qR;
    side_state<float, CURVED, 0, true, true>(fL, mf, (float)gam, (float)gfac, sL, mf.ia);
    side_state<float, CURVED, 0, true, true>(fR, mf, (float)gam, (float)gfac, sR, mf.ia);
    side_states_x2<CURVED>(fL, fR, mf, (float)gam, (float)gfac, mf.ia, qL, qR);
    atomicAdd(cnt + 1, 1ull);
    const Side<float>* P[2] = {&qL, &qR};
    const Side<float>* S[2] = {&sL, &sR};
    const Side<double>* D[2] = {&dL, &dR};
    for (int s = 0; s < 2; ++s) {
      const double spd[2] = {D[s]->lp, D[s]->lm};
      const float ps[2] = {P[s]->lp, P[s]->lm}, ss[2] = {S[s]->lp, S[s]->lm};
      const float e[8] = {err(P[s]->U, D[s]->U, 8), err(P[s]->F, D[s]->F, 8), err(ps, spd, 2),
                          err(&P[s]->sden, &D[s]->sden, 1), err(S[s]->U, D[s]->U, 8), err(S[s]->F, D[s]->F, 8),
                          err(ss, spd, 2), err(&S[s]->sden, &D[s]->sden, 1)};
      for (int k = 0; k < 8; ++k) atomicMax(reinterpret_cast<unsigned int*>(out + k), __float_as_uint(e[k]));
    }
  }
}

int main() {
  const long long n = 1ll << 20;
  float* out;
  unsigned long long* cnt;
  if (cudaMalloc(&out, 16 * sizeof(float)) != cudaSuccess || cudaMalloc(&cnt, 4 * sizeof(unsigned long long)) != cudaSuccess)
    return 2;
  int rc = 0;
  for (int curved = 0; curved < 2; ++curved) {
    cudaMemset(out, 0, 16 * sizeof(float));
    cudaMemset(cnt, 0, 4 * sizeof(unsigned long long));
    if (curved) check<true><<<152 * 4, 256>>>(n, out, cnt);
    else check<false><<<152 * 4, 256>>>(n, out, cnt);
    float h[8];
    unsigned long long c[2];
    cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
    cudaMemcpy(c, cnt, sizeof(c), cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = 1;
    printf("%d %llu %llu %.3e %.3e %.3e %.3e %.3e %.3e %.3e %.3e %s\n", curved, c[0], c[1], h[0], h[1], h[2], h[3], h[4],
           h[5], h[6], h[7], e == cudaSuccess ? "ok" : cudaGetErrorString(e));
  }
  cudaFree(out);
  cudaFree(cnt);
  return rc;
}
"""


@pytest.mark.gpu
def test_paired_side_states_are_as_accurate_as_the_scalar_form(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "check.cu"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC, "-I",
                    INCLUDE, str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout.split("\n")
    rows = [ln.split() for ln in lines if ln.strip()]
    assert len(rows) == 2, lines
    for r in rows:
        assert r[-1] == "ok", r
        assert int(r[1]) == 0, f"paired physical-state checks differ from physical_state<float>: {r}"
        assert int(r[2]) == 1 << 20
        paired, scalar = [float(x) for x in r[3:7]], [float(x) for x in r[7:11]]
        for a, b in zip(paired, scalar):
            assert a <= max(2.0 * b, 1e-6), (r, paired, scalar)
            assert a <= 1e-4, (r, paired)
