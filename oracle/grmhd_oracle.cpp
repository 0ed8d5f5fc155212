// GRMHD oracle: a plain, slow, FP64 CPU implementation of the Valencia
// method-of-lines hot path of GRaM-X (arXiv 2210.17509).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
// load or call this file.  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg use it.  It shares no code, header, table or
// constant with the CUDA library; the two meet only through plain arrays.
//
// The oracle follows the paper's equations in their covariant form, which is
// deliberately different from the 3+1 component formulas the CUDA kernels use:
//   * conserved variables and fluxes are projections of the conserved
//     currents J^mu = rho u^mu, T^{mu nu} (Eq. 5) and the dual Faraday tensor
//     *F^{mu nu} = u^mu b^nu - u^nu b^mu, multiplied by sqrt(-g); this
//     reproduces Eqs. 6-9 (prim -> cons) and Eq. 12 (flux) of Sec. 2.2;
//   * source terms are Eq. 13 written with the 4-Christoffel symbols of the
//     4-metric assembled from (alpha, beta^i, gamma_ij) (Sec. 2.1 lists these
//     ADM variables as the interface to the hydrodynamics);
//   * wave speeds are the roots of the covariant fast-magnetosonic quadratic;
//   * con2prim (Sec. 2.3, recovery step) is a 1D bracketed bisection in
//     z = rho h W^2, followed by one Newton polish; the CUDA path uses a 2D
//     Newton-Raphson in (z, W).
// Every routine is templated on the scalar so that a forward-mode dual number
// gives directional derivatives of the whole evolution.
//
// Readings of the paper that the text leaves open (all shared with the CUDA
// path because the method itself depends on them):
//   R1 reconstructed primitives are [rho, v^x, v^y, v^z, P, B^x, B^y, B^z];
//   R2 minmod slope, tie -> first argument; face value = centre +- slope/2;
//   R3 WENO5 = Jiang-Shu indicators, linear weights (1/10, 6/10, 3/10),
//      alpha_k = d_k / (eps + beta_k)^2 with eps a parameter (default 1e-6);
//   R4 all 8 components go through HLLE, no constrained transport;
//   R5 HLLE signal speeds from a^2 = cs^2 + vA^2 - cs^2 vA^2 (Sec. 2.3 cites
//      Gammie 2003), xi- = min(0, lm_L, lm_R), xi+ = max(0, lp_L, lp_R);
//      if xi+ - xi- < 1e-300 the flux is the mean of the two physical fluxes;
//   R6 b^mu = (B^mu + (u_nu B^nu) u^mu) / W with B^mu = (0, B^i);
//   R7 metric given at cell centres; face value = mean of the two cells;
//      metric derivatives by 4th-order centred differences; the time
//      derivative of gamma_ij follows from K_ij with static lapse and shift;
//   R8 Gamma-law EOS P = (Gamma - 1) rho eps (Sec. 2.3);
//   R9 boundary: periodic, or copy of the nearest interior primitive;
//   R10 RK2 = SSP Heun, RK3 = SSP Shu-Osher, RK4 = classical; every stage is
//      con2prim -> ghost fill -> RHS (the RHS recipe of Sec. 2.3);
//   R11 a reconstructed face state with rho <= 0, P <= 0 or v^2 >= 1 (one of
//      the unphysical outcomes Sec. 2.3 lists for the recovery) is replaced
//      by the primitive state of the cell it was reconstructed from;
//   R12 recovery failures (Sec. 2.3 lists them): no root, NaN, rho < rho_atm
//      or v >= 1 -> atmosphere (rho_atm, v = 0, p_atm, B kept); a root with
//      P <= 0 but valid rho and v -> pressure floor P = p_atm.  "No root"
//      includes the case where the energy residual has no sign change
//      inside v < 1: a bracket that closes only against the v = 1 boundary
//      is not a root (its side of the boundary is decided by round-off).
//   R18 Newman-Hamlin recovery (Sec. 2.3: an effective 1D iteration over the
//      pressure; each step solves a cubic in eps = B^2 + z): from the energy
//      and momentum equations, eps^3 - a eps^2 + d = 0 with a = tau + D + P
//      + B^2 / 2 and d = (B^2 S^2 - (B.S)^2) / 2; the physical root is the
//      largest, eps = a/3 + (2a/3) cos(acos(1 - 27 d / (2 a^3)) / 3); then
//      z = eps - B^2, v^2(z) from the momentum equation, and the Gamma-law
//      pressure of (z, W) is the next iterate.  Plain fixed point here; the
//      GPU path accelerates it (Aitken) and uses it as the fallback of its
//      Newton iteration.
//   R19 constrained transport (Sec. 3, staggered grids: the vector potential
//      on cell edges keeps div B zero to round-off; used by the rotor and
//      explosion tests and the TOV star): the densitised field lives on cell
//      faces (component a on the a-faces) and is the discrete curl of an
//      edge potential at the start; every stage changes it by minus the
//      discrete curl of the edge electric field E, each E_c the mean of the
//      four face fluxes of the field around its edge (E_c = -F_a(B^b) =
//      F_b(B^a) for (c, a, b) cyclic; Balsara & Spicer's averaging).  The
//      cell-centred field that the rest of the scheme sees is the mean of
//      the two faces along its direction.
//   R20 polytropic EOS (Sec. 2.3, EOS paragraph: P = K rho^Gamma, with the
//      atmosphere pressure from the same polytrope as in Sec. 4.4): the
//      pressure is a function of the density everywhere it is used (cell
//      states, the reconstructed face states, prim -> cons), eps = P /
//      ((Gamma - 1) rho) as for the Gamma-law, and the recovery uses D, S_i
//      and B^i only (tau is evolved but not read): with rho = D / W, z =
//      rho h W^2 is a function of W, and the momentum equation
//      (z + B^2)^2 (1 - 1/W^2) - (B.S)^2 (2z + B^2) / z^2 = S^2 is solved
//      for W >= 1 by bisection (its left side is 0 - (B.S)^2 (...) <= S^2
//      at W = 1 and grows without bound).  The atmosphere is rho_atm, v = 0,
//      P = K rho_atm^Gamma.
//   Two-level block AMR without subcycling (Sec. 3: refined grids halve the
//   spacing, are properly nested, share one global time step; ghost zones
//   of a refined grid are filled by prolongation from the next coarser
//   level, covered coarse cells are reset by restriction, fine fluxes are
//   restricted onto the coarse grid):
//   R14 restriction acts on the conserved variables: a covered coarse cell
//      becomes the mean of its 8 children (equal coordinate volumes, so the
//      mean conserves the integral).
//   R15 prolongation acts on the primitives (the ghost zones hold
//      primitives, R9): a fine point takes its coarse parent's value plus,
//      per axis, the parent's minmod-limited slope (R2) times the child's
//      offset of -1/4 or +1/4 coarse cell; the 8 children average to the
//      parent.  The paper names high-order operators without an order.
//   R16 flux restriction: on every coarse face of the coarse-fine
//      interface, the uncovered coarse cell's RHS uses the mean of the 4
//      fine face fluxes instead of the coarse face flux (one global dt, so no
//      time integration of fluxes, "refluxing", is needed).
//   R17 composite stage: RHS of every block -> flux restriction onto the
//      coarse RHS -> stage update -> restriction of the fine U -> recovery on
//      every block -> coarse ghosts by its boundary condition, fine ghosts by
//      prolongation from the coarse primitives.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ---------------------------------------------------------------- scalars --
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
};

inline double val(double x) { return x; }
template <int N> inline double val(const Dual<N>& x) { return x.v; }

template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r; r.v = a.v * b; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r;
}
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }
template <int N> inline Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { a = a - b; return a; }
template <int N> inline Dual<N>& operator*=(Dual<N>& a, const Dual<N>& b) { a = a * b; return a; }
template <int N> inline Dual<N>& operator/=(Dual<N>& a, const Dual<N>& b) { a = a / b; return a; }
template <int N> inline bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N> inline bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }
template <int N> inline bool operator<=(const Dual<N>& a, const Dual<N>& b) { return a.v <= b.v; }
template <int N> inline bool operator>=(const Dual<N>& a, const Dual<N>& b) { return a.v >= b.v; }
template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v);
  const double s = (r.v > 0.0) ? 0.5 / r.v : 0.0;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
  return r;
}
template <int N> inline Dual<N> fabs(const Dual<N>& a) { return (a.v < 0.0) ? -a : a; }
template <int N> inline Dual<N> pow(const Dual<N>& a, double e) {
  Dual<N> r; r.v = std::pow(a.v, e);
  const double s = e * std::pow(a.v, e - 1.0);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
  return r;
}
using std::sqrt;
using std::fabs;

template <class S> inline S smin(const S& a, const S& b) { return (b < a) ? b : a; }
template <class S> inline S smax(const S& a, const S& b) { return (a < b) ? b : a; }
template <class S> inline S sq(const S& a) { return a * a; }

// ------------------------------------------------------------------- grid --
struct Grid {
  int n[3];
  int ng;
  double dx[3];
  int N[3];
  long ncell;
  void init(const int* n3, int ng_, const double* dx3) {
    for (int d = 0; d < 3; ++d) { n[d] = n3[d]; dx[d] = dx3[d]; N[d] = n3[d] + 2 * ng_; }
    ng = ng_;
    ncell = (long)N[0] * N[1] * N[2];
  }
  long at(int i, int j, int k) const { return ((long)k * N[1] + j) * N[0] + i; }
  bool interior(int i, int j, int k) const {
    return i >= ng && i < ng + n[0] && j >= ng && j < ng + n[1] && k >= ng && k < ng + n[2];
  }
};

enum { REC_MINMOD = 0, REC_WENO5 = 1 };
enum { BC_PERIODIC = 0, BC_COPY = 1 };
enum { RK2 = 2, RK3 = 3, RK4 = 4 };

// Oracle-side parameter block (plain C layout, mirrored by the Python wrapper).
struct OParams {
  double gamma;     // adiabatic index (Sec. 2.3, EOS paragraph)
  int32_t recon;    // REC_MINMOD | REC_WENO5
  int32_t bc;       // BC_PERIODIC | BC_COPY
  double rho_atm;   // atmosphere density floor (Sec. 4.4 uses an atmosphere)
  double p_atm;     // atmosphere pressure (Gamma-law)
  double weno_eps;  // WENO5 epsilon (reading R3)
  int32_t eos;      // EOS_IDEAL (Gamma-law) | EOS_POLYTROPE (reading R20)
  double poly_K;    // polytropic constant K of P = K rho^Gamma
};

enum { EOS_IDEAL = 0, EOS_POLYTROPE = 1 };

template <class S>
struct Par {
  S gamma;
  int recon, bc;
  double rho_atm, p_atm, weno_eps;
  int eos = EOS_IDEAL;
  double poly_K = 0.0;
};

// Reading R20: under the polytrope the pressure entry of a primitive state
// is K rho^Gamma (states with rho <= 0 are left for the caller's checks).
template <class S>
void apply_eos(const Par<S>& p, S pr[8]) {
  using std::pow;
  if (p.eos == EOS_POLYTROPE && val(pr[0]) > 0.0) pr[4] = p.poly_K * pow(pr[0], val(p.gamma));
}

// --------------------------------------------------- 4-metric (Sec. 2.1) --
// ADM component order in every metric array: alpha, beta^x, beta^y, beta^z,
// gamma_xx, gamma_xy, gamma_xz, gamma_yy, gamma_yz, gamma_zz.
static const int SYM[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};

// Gauss-Jordan inverse with partial pivoting; returns the determinant.
template <class S, int M>
S invert_gj(const S a_in[M][M], S inv[M][M]) {
  S a[M][M];
  for (int r = 0; r < M; ++r)
    for (int c = 0; c < M; ++c) { a[r][c] = a_in[r][c]; inv[r][c] = S(r == c ? 1.0 : 0.0); }
  S det = S(1.0);
  for (int c = 0; c < M; ++c) {
    int p = c;
    for (int r = c + 1; r < M; ++r)
      if (std::fabs(val(a[r][c])) > std::fabs(val(a[p][c]))) p = r;
    if (p != c) {
      for (int k = 0; k < M; ++k) { std::swap(a[p][k], a[c][k]); std::swap(inv[p][k], inv[c][k]); }
      det = -det;
    }
    const S piv = a[c][c];
    det = det * piv;
    const S ip = S(1.0) / piv;
    for (int k = 0; k < M; ++k) { a[c][k] = a[c][k] * ip; inv[c][k] = inv[c][k] * ip; }
    for (int r = 0; r < M; ++r) {
      if (r == c) continue;
      const S f = a[r][c];
      if (val(f) == 0.0) continue;
      for (int k = 0; k < M; ++k) { a[r][k] = a[r][k] - f * a[c][k]; inv[r][k] = inv[r][k] - f * inv[c][k]; }
    }
  }
  return det;
}

template <class S>
struct Spacetime {
  S alpha, beta[3], gam[3][3];
  S g[4][4], gu[4][4];   // g_{mu nu}, g^{mu nu}
  S sqrtmg, sqrtgam;     // sqrt(-g), sqrt(gamma)
};

template <class S>
void spacetime_from_adm(const S adm[10], Spacetime<S>& st) {
  st.alpha = adm[0];
  for (int i = 0; i < 3; ++i) st.beta[i] = adm[1 + i];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) st.gam[i][j] = adm[SYM[i][j]];
  S betal[3];
  for (int i = 0; i < 3; ++i) {
    betal[i] = S(0.0);
    for (int j = 0; j < 3; ++j) betal[i] += st.gam[i][j] * st.beta[j];
  }
  S b2 = S(0.0);
  for (int i = 0; i < 3; ++i) b2 += betal[i] * st.beta[i];
  st.g[0][0] = b2 - st.alpha * st.alpha;
  for (int i = 0; i < 3; ++i) { st.g[0][1 + i] = betal[i]; st.g[1 + i][0] = betal[i]; }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) st.g[1 + i][1 + j] = st.gam[i][j];
  const S detg = invert_gj<S, 4>(st.g, st.gu);
  st.sqrtmg = sqrt(-detg);
  st.sqrtgam = st.sqrtmg / st.alpha;
}

template <class S>
void flat_adm(S adm[10]) {
  for (int c = 0; c < 10; ++c) adm[c] = S(0.0);
  adm[0] = S(1.0); adm[4] = S(1.0); adm[7] = S(1.0); adm[9] = S(1.0);
}

// --------------------------------------------- fluid state (Sec. 2.2) --
template <class S>
struct Fluid {
  S rho, press, v[3], B[3];       // primitives; v^i Valencia (Eq. 10), B^i Eulerian
  S W, u[4], ul[4], b[4], b2, h, rhohs, ps;
  S T[4][4];                      // T^{mu nu}, Eq. 5
  S Fd[4][4];                     // dual Faraday *F^{mu nu}
  S J[4];                         // rest-mass current rho u^mu
};

template <class S>
void fluid_from_prim(const S p[8], const Spacetime<S>& st, const S& gamma, Fluid<S>& f) {
  f.rho = p[0];
  for (int i = 0; i < 3; ++i) f.v[i] = p[1 + i];
  f.press = p[4];
  for (int i = 0; i < 3; ++i) f.B[i] = p[5 + i];
  S v2 = S(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) v2 += st.gam[i][j] * f.v[i] * f.v[j];
  f.W = S(1.0) / sqrt(S(1.0) - v2);
  // Eq. 10 inverted: u^i = W (v^i - beta^i / alpha), u^0 = W / alpha.
  f.u[0] = f.W / st.alpha;
  for (int i = 0; i < 3; ++i) f.u[1 + i] = f.W * (f.v[i] - st.beta[i] / st.alpha);
  for (int m = 0; m < 4; ++m) {
    f.ul[m] = S(0.0);
    for (int n = 0; n < 4; ++n) f.ul[m] += st.g[m][n] * f.u[n];
  }
  // Reading R6: b^mu = (B^mu + (u_nu B^nu) u^mu) / W, B^mu = (0, B^i).
  S uB = S(0.0);
  for (int i = 0; i < 3; ++i) uB += f.ul[1 + i] * f.B[i];
  f.b[0] = uB * f.u[0] / f.W;
  for (int i = 0; i < 3; ++i) f.b[1 + i] = (f.B[i] + uB * f.u[1 + i]) / f.W;
  f.b2 = S(0.0);
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) f.b2 += st.g[m][n] * f.b[m] * f.b[n];
  // Gamma-law: eps = P / ((Gamma - 1) rho); h = 1 + eps + P / rho (Sec. 2.2/2.3).
  const S eps = f.press / ((gamma - 1.0) * f.rho);
  f.h = S(1.0) + eps + f.press / f.rho;
  f.rhohs = f.rho * f.h + f.b2;           // rho h*
  f.ps = f.press + 0.5 * f.b2;            // P* = P + b^2 / 2
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) {
      f.T[m][n] = f.rhohs * f.u[m] * f.u[n] + f.ps * st.gu[m][n] - f.b[m] * f.b[n];
      f.Fd[m][n] = f.u[m] * f.b[n] - f.u[n] * f.b[m];
    }
  for (int m = 0; m < 4; ++m) f.J[m] = f.rho * f.u[m];
}

// Conserved vector U = [D, S_j, tau, B~^k] as projections of the currents
// (equivalent to Eqs. 6-9): D = sqrt(-g) J^0, S_j = sqrt(-g) T^0_j,
// tau = sqrt(-g) (alpha T^00 - J^0), B~^k = -sqrt(-g) *F^{k0}.
template <class S>
void conserved(const Fluid<S>& f, const Spacetime<S>& st, S U[8]) {
  const S s = st.sqrtmg;
  U[0] = s * f.J[0];
  for (int j = 0; j < 3; ++j) {
    S t = S(0.0);
    for (int m = 0; m < 4; ++m) t += f.T[0][m] * st.g[m][1 + j];
    U[1 + j] = s * t;
  }
  U[4] = s * (st.alpha * f.T[0][0] - f.J[0]);
  for (int k = 0; k < 3; ++k) U[5 + k] = -s * f.Fd[1 + k][0];
}

// Flux F^i in direction d (equivalent to Eq. 12): sqrt(-g) [J^i, T^i_j,
// alpha T^{0i} - J^i, *F^{ik}].
template <class S>
void flux(const Fluid<S>& f, const Spacetime<S>& st, int d, S F[8]) {
  const int i = 1 + d;
  const S s = st.sqrtmg;
  F[0] = s * f.J[i];
  for (int j = 0; j < 3; ++j) {
    S t = S(0.0);
    for (int m = 0; m < 4; ++m) t += f.T[i][m] * st.g[m][1 + j];
    F[1 + j] = s * t;
  }
  F[4] = s * (st.alpha * f.T[0][i] - f.J[i]);
  for (int k = 0; k < 3; ++k) F[5 + k] = s * f.Fd[i][1 + k];
}

// Reading R5: signal speeds dx^d/dt = lambda solve
// (1 - a^2)(k.u)^2 = a^2 k.k for the covector k = (-lambda, e_d).
template <class S>
void wave_speeds(const Fluid<S>& f, const Spacetime<S>& st, const S& gamma, int d, S& lm, S& lp) {
  const int i = 1 + d;
  const S cs2 = gamma * f.press / (f.rho * f.h);
  const S va2 = f.b2 / (f.rho * f.h + f.b2);
  const S a2 = cs2 + va2 - cs2 * va2;
  const S A = (1.0 - a2) * f.u[0] * f.u[0] - a2 * st.gu[0][0];
  const S B = -2.0 * ((1.0 - a2) * f.u[0] * f.u[i] - a2 * st.gu[0][i]);
  const S C = (1.0 - a2) * f.u[i] * f.u[i] - a2 * st.gu[i][i];
  S disc = B * B - 4.0 * A * C;
  S sd = (val(disc) > 0.0) ? sqrt(disc) : S(0.0);
  const S r1 = (-B + sd) / (2.0 * A);
  const S r2 = (-B - sd) / (2.0 * A);
  lp = smax(r1, r2);
  lm = smin(r1, r2);
}

// ------------------------------------------------------- reconstruction --
template <class S>
S minmod(const S& a, const S& b) {
  if (val(a) * val(b) <= 0.0) return S(0.0);
  return (std::fabs(val(a)) <= std::fabs(val(b))) ? a : b;
}

// Jiang-Shu WENO5 value at the right face i+1/2 of cell i from the five cell
// values i-2 .. i+2 (Shu 1998, cited in Sec. 2.3).
template <class S>
S weno5_right_face(const S& um2, const S& um1, const S& u0, const S& up1, const S& up2, double eps) {
  const S q0 = (2.0 * um2 - 7.0 * um1 + 11.0 * u0) / 6.0;
  const S q1 = (-1.0 * um1 + 5.0 * u0 + 2.0 * up1) / 6.0;
  const S q2 = (2.0 * u0 + 5.0 * up1 - up2) / 6.0;
  const S b0 = (13.0 / 12.0) * sq(um2 - 2.0 * um1 + u0) + 0.25 * sq(um2 - 4.0 * um1 + 3.0 * u0);
  const S b1 = (13.0 / 12.0) * sq(um1 - 2.0 * u0 + up1) + 0.25 * sq(um1 - up1);
  const S b2 = (13.0 / 12.0) * sq(u0 - 2.0 * up1 + up2) + 0.25 * sq(3.0 * u0 - 4.0 * up1 + up2);
  const S a0 = 0.1 / sq(eps + b0);
  const S a1 = 0.6 / sq(eps + b1);
  const S a2 = 0.3 / sq(eps + b2);
  const S sum = a0 + a1 + a2;
  return (a0 / sum) * q0 + (a1 / sum) * q1 + (a2 / sum) * q2;
}

// The two states at the face between cells c-1 and c from the six values
// u[0..5] = cells c-3 .. c+2.  uL comes from cell c-1, uR from cell c.
template <class S>
void reconstruct_face(int recon, double eps, const S u[6], S& uL, S& uR) {
  if (recon == REC_MINMOD) {
    uL = u[2] + 0.5 * minmod(u[2] - u[1], u[3] - u[2]);
    uR = u[3] - 0.5 * minmod(u[3] - u[2], u[4] - u[3]);
  } else {
    uL = weno5_right_face(u[0], u[1], u[2], u[3], u[4], eps);
    uR = weno5_right_face(u[5], u[4], u[3], u[2], u[1], eps);
  }
}

// ------------------------------------------------------------------ HLLE --
template <class S>
struct FaceOut {
  S F[8];
  S lmL, lpL, lmR, lpR;
};

template <class S>
void hlle(const S pL[8], const S pR[8], const S adm[10], const S& gamma, int d, FaceOut<S>& out) {
  Spacetime<S> st;
  spacetime_from_adm(adm, st);
  Fluid<S> fL, fR;
  fluid_from_prim(pL, st, gamma, fL);
  fluid_from_prim(pR, st, gamma, fR);
  S UL[8], UR[8], FL[8], FR[8];
  conserved(fL, st, UL);
  conserved(fR, st, UR);
  flux(fL, st, d, FL);
  flux(fR, st, d, FR);
  wave_speeds(fL, st, gamma, d, out.lmL, out.lpL);
  wave_speeds(fR, st, gamma, d, out.lmR, out.lpR);
  const S xm = smin(S(0.0), smin(out.lmL, out.lmR));
  const S xp = smax(S(0.0), smax(out.lpL, out.lpR));
  if (val(xp) - val(xm) < 1e-300) {
    for (int c = 0; c < 8; ++c) out.F[c] = 0.5 * (FL[c] + FR[c]);
    return;
  }
  for (int c = 0; c < 8; ++c)
    out.F[c] = (xp * FL[c] - xm * FR[c] + xp * xm * (UR[c] - UL[c])) / (xp - xm);
}

// --------------------------------------------------------- block helpers --
template <class S>
void load_adm(const Grid& G, const double* metric, long c, S adm[10]) {
  if (!metric) { flat_adm(adm); return; }
  for (int q = 0; q < 10; ++q) adm[q] = S(metric[q * G.ncell + c]);
}

// Flux through the face between cell (i,j,k) - e_d and cell (i,j,k).
template <class S>
void face_flux(const Grid& G, const Par<S>& p, const S* prim, const double* metric,
               int d, int i, int j, int k, S F[8]) {
  int off[3] = {0, 0, 0};
  S pL[8], pR[8];
  for (int q = 0; q < 8; ++q) {
    S u[6];
    for (int s = 0; s < 6; ++s) {
      off[d] = s - 3;
      u[s] = prim[q * G.ncell + G.at(i + off[0], j + off[1], k + off[2])];
    }
    off[d] = 0;
    reconstruct_face(p.recon, p.weno_eps, u, pL[q], pR[q]);
  }
  off[d] = -1;
  const long cm = G.at(i + off[0], j + off[1], k + off[2]), cp = G.at(i, j, k);
  S a0[10], a1[10], adm[10];
  load_adm(G, metric, cm, a0);
  load_adm(G, metric, cp, a1);
  for (int q = 0; q < 10; ++q) adm[q] = 0.5 * (a0[q] + a1[q]);
  // Reading R11: unphysical face states fall back to their cell's state.
  auto physical = [&](const S pr[8]) {
    double v2 = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) v2 += val(adm[SYM[a][b]]) * val(pr[1 + a]) * val(pr[1 + b]);
    return val(pr[0]) > 0.0 && val(pr[4]) > 0.0 && v2 < 1.0;
  };
  // Reading R20: a polytrope's face pressure follows from the face density.
  apply_eos(p, pL);
  apply_eos(p, pR);
  if (!physical(pL)) {
    for (int q = 0; q < 8; ++q) pL[q] = prim[q * G.ncell + cm];
    apply_eos(p, pL);
  }
  if (!physical(pR)) {
    for (int q = 0; q < 8; ++q) pR[q] = prim[q * G.ncell + cp];
    apply_eos(p, pR);
  }
  FaceOut<S> fo;
  hlle(pL, pR, adm, p.gamma, d, fo);
  for (int q = 0; q < 8; ++q) F[q] = fo.F[q];
}

// 4th-order centred derivative of ADM component q along direction e.
inline double fd4(const Grid& G, const double* metric, int q, int e, int i, int j, int k) {
  int o[3] = {0, 0, 0};
  double f[5];
  for (int s = -2; s <= 2; ++s) {
    o[e] = s;
    f[s + 2] = metric[q * G.ncell + G.at(i + o[0], j + o[1], k + o[2])];
  }
  return (-f[4] + 8.0 * f[3] - 8.0 * f[1] + f[0]) / (12.0 * G.dx[e]);
}

// Eq. 13 source terms at the centre of cell (i,j,k), covariant form.
template <class S>
void source_cell(const Grid& G, const Par<S>& p, const S* prim, const double* metric,
                 const double* Kij, int i, int j, int k, S src[8]) {
  for (int q = 0; q < 8; ++q) src[q] = S(0.0);
  if (!metric) return;  // Minkowski: all Christoffels and derivatives vanish
  const long c = G.at(i, j, k);
  double adm[10];
  for (int q = 0; q < 10; ++q) adm[q] = metric[q * G.ncell + c];
  Spacetime<double> st;
  spacetime_from_adm(adm, st);
  // dA[e][q]: spatial derivative (e = 0..2) of ADM component q.
  double dA[3][10];
  for (int e = 0; e < 3; ++e)
    for (int q = 0; q < 10; ++q) dA[e][q] = fd4(G, metric, q, e, i, j, k);
  double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (Kij)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) K[a][b] = Kij[(SYM[a][b] - 4) * G.ncell + c];
  // dg[mu][a][b] = d_mu g_ab (mu = 0 time).
  double dg[4][4][4];
  const double* beta = st.beta;
  double betal[3];
  for (int a = 0; a < 3; ++a) {
    betal[a] = 0.0;
    for (int b = 0; b < 3; ++b) betal[a] += st.gam[a][b] * beta[b];
  }
  for (int e = 0; e < 3; ++e) {
    double dgam[3][3], dbeta[3];
    for (int a = 0; a < 3; ++a) {
      dbeta[a] = dA[e][1 + a];
      for (int b = 0; b < 3; ++b) dgam[a][b] = dA[e][SYM[a][b]];
    }
    double d00 = -2.0 * st.alpha * dA[e][0];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) d00 += dgam[a][b] * beta[a] * beta[b] + 2.0 * st.gam[a][b] * beta[a] * dbeta[b];
    dg[1 + e][0][0] = d00;
    for (int a = 0; a < 3; ++a) {
      double t = 0.0;
      for (int b = 0; b < 3; ++b) t += dgam[a][b] * beta[b] + st.gam[a][b] * dbeta[b];
      dg[1 + e][0][1 + a] = t;
      dg[1 + e][1 + a][0] = t;
      for (int b = 0; b < 3; ++b) dg[1 + e][1 + a][1 + b] = dgam[a][b];
    }
  }
  // d_t gamma_ab = -2 alpha K_ab + beta^m d_m gamma_ab + gamma_mb d_a beta^m + gamma_am d_b beta^m
  double dtgam[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double t = -2.0 * st.alpha * K[a][b];
      for (int m = 0; m < 3; ++m)
        t += beta[m] * dA[m][SYM[a][b]] + st.gam[m][b] * dA[a][1 + m] + st.gam[a][m] * dA[b][1 + m];
      dtgam[a][b] = t;
    }
  {
    double d00 = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) d00 += dtgam[a][b] * beta[a] * beta[b];
    dg[0][0][0] = d00;
    for (int a = 0; a < 3; ++a) {
      double t = 0.0;
      for (int b = 0; b < 3; ++b) t += dtgam[a][b] * beta[b];
      dg[0][0][1 + a] = t;
      dg[0][1 + a][0] = t;
      for (int b = 0; b < 3; ++b) dg[0][1 + a][1 + b] = dtgam[a][b];
    }
  }
  // 4-Christoffel symbols Gamma^l_{mn} = 1/2 g^{ls} (d_m g_sn + d_n g_sm - d_s g_mn).
  double Chr[4][4][4];
  for (int l = 0; l < 4; ++l)
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) {
        double t = 0.0;
        for (int s = 0; s < 4; ++s) t += st.gu[l][s] * (dg[m][s][n] + dg[n][s][m] - dg[s][m][n]);
        Chr[l][m][n] = 0.5 * t;
      }
  S pc[8];
  for (int q = 0; q < 8; ++q) pc[q] = prim[q * G.ncell + c];
  apply_eos(p, pc);
  Spacetime<S> sts;
  S admS[10];
  for (int q = 0; q < 10; ++q) admS[q] = S(adm[q]);
  spacetime_from_adm(admS, sts);
  Fluid<S> f;
  fluid_from_prim(pc, sts, p.gamma, f);
  const double smg = st.sqrtmg;
  // momentum: sqrt(-g) T^{mn} (d_m g_{nj} - Gamma^l_{mn} g_{lj})
  for (int jj = 0; jj < 3; ++jj) {
    S t = S(0.0);
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) {
        double w = dg[m][n][1 + jj];
        for (int l = 0; l < 4; ++l) w -= Chr[l][m][n] * st.g[l][1 + jj];
        t += f.T[m][n] * w;
      }
    src[1 + jj] = smg * t;
  }
  // energy: sqrt(-g) alpha (T^{m0} d_m ln alpha - T^{mn} Gamma^0_{mn}); d_t alpha = 0.
  {
    S t = S(0.0);
    for (int e = 0; e < 3; ++e) t += f.T[1 + e][0] * (dA[e][0] / st.alpha);
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) t -= f.T[m][n] * Chr[0][m][n];
    src[4] = smg * st.alpha * t;
  }
}

// Method-of-lines right-hand side dU/dt = -d_i F^i + S (Eq. 11), on the
// interior; ghost entries of rhs are set to zero.  Face fluxes are stored
// explicitly and the divergence is summed in x, y, z order.
template <class S>
void rhs_block(const Grid& G, const Par<S>& p, const S* prim, const double* metric,
               const double* Kij, S* rhs) {
  for (long c = 0; c < 8 * G.ncell; ++c) rhs[c] = S(0.0);
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2], g = G.ng;
  std::vector<S> Fx((size_t)8 * (nx + 1) * ny * nz), Fy((size_t)8 * nx * (ny + 1) * nz),
      Fz((size_t)8 * nx * ny * (nz + 1));
  auto ix = [&](int a, int b, int c2) { return ((size_t)c2 * ny + b) * (nx + 1) + a; };
  auto iy = [&](int a, int b, int c2) { return ((size_t)c2 * (ny + 1) + b) * nx + a; };
  auto iz = [&](int a, int b, int c2) { return ((size_t)c2 * ny + b) * nx + a; };
#pragma omp parallel for schedule(dynamic, 1)
  for (int kk = 0; kk < nz + 1; ++kk) {
    S F[8];
    for (int jj = 0; jj < ny + 1; ++jj)
      for (int ii = 0; ii < nx + 1; ++ii) {
        if (jj < ny && kk < nz) {
          face_flux(G, p, prim, metric, 0, g + ii, g + jj, g + kk, F);
          for (int q = 0; q < 8; ++q) Fx[q * (size_t)(nx + 1) * ny * nz + ix(ii, jj, kk)] = F[q];
        }
        if (ii < nx && kk < nz) {
          face_flux(G, p, prim, metric, 1, g + ii, g + jj, g + kk, F);
          for (int q = 0; q < 8; ++q) Fy[q * (size_t)nx * (ny + 1) * nz + iy(ii, jj, kk)] = F[q];
        }
        if (ii < nx && jj < ny) {
          face_flux(G, p, prim, metric, 2, g + ii, g + jj, g + kk, F);
          for (int q = 0; q < 8; ++q) Fz[q * (size_t)nx * ny * (nz + 1) + iz(ii, jj, kk)] = F[q];
        }
      }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int kk = 0; kk < nz; ++kk)
    for (int jj = 0; jj < ny; ++jj)
      for (int ii = 0; ii < nx; ++ii) {
        const long c = G.at(g + ii, g + jj, g + kk);
        S src[8];
        source_cell(G, p, prim, metric, Kij, g + ii, g + jj, g + kk, src);
        for (int q = 0; q < 8; ++q) {
          const size_t sx = q * (size_t)(nx + 1) * ny * nz;
          const size_t sy = q * (size_t)nx * (ny + 1) * nz;
          const size_t sz = q * (size_t)nx * ny * (nz + 1);
          S r = S(0.0);
          r = r - (Fx[sx + ix(ii + 1, jj, kk)] - Fx[sx + ix(ii, jj, kk)]) / G.dx[0];
          r = r - (Fy[sy + iy(ii, jj + 1, kk)] - Fy[sy + iy(ii, jj, kk)]) / G.dx[1];
          r = r - (Fz[sz + iz(ii, jj, kk + 1)] - Fz[sz + iz(ii, jj, kk)]) / G.dx[2];
          rhs[q * G.ncell + c] = r + src[q];
        }
      }
}

// RHS of single cells (for spot checks of large blocks).
template <class S>
void rhs_one_cell(const Grid& G, const Par<S>& p, const S* prim, const double* metric,
                  const double* Kij, int i, int j, int k, S out[8]) {
  S lo[8], hi[8], src[8];
  for (int q = 0; q < 8; ++q) out[q] = S(0.0);
  for (int d = 0; d < 3; ++d) {
    int o[3] = {0, 0, 0};
    o[d] = 1;
    face_flux(G, p, prim, metric, d, i, j, k, lo);
    face_flux(G, p, prim, metric, d, i + o[0], j + o[1], k + o[2], hi);
    for (int q = 0; q < 8; ++q) out[q] = out[q] - (hi[q] - lo[q]) / G.dx[d];
  }
  source_cell(G, p, prim, metric, Kij, i, j, k, src);
  for (int q = 0; q < 8; ++q) out[q] = out[q] + src[q];
}

// -------------------------------------------------- prim -> cons (Eq. 6-9) --
template <class S>
void prim2con_block(const Grid& G, const S& gamma, const S* prim, const double* metric, S* cons,
                    int eos = EOS_IDEAL, double poly_K = 0.0) {
  Par<S> pe;
  pe.gamma = gamma;
  pe.eos = eos;
  pe.poly_K = poly_K;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < G.ncell; ++c) {
    S adm[10], p[8], U[8];
    load_adm(G, metric, c, adm);
    Spacetime<S> st;
    spacetime_from_adm(adm, st);
    for (int q = 0; q < 8; ++q) p[q] = prim[q * G.ncell + c];
    apply_eos(pe, p);
    Fluid<S> f;
    fluid_from_prim(p, st, gamma, f);
    conserved(f, st, U);
    for (int q = 0; q < 8; ++q) cons[q * G.ncell + c] = U[q];
  }
}

// ------------------------------------------------ con2prim (Sec. 2.3) --
// Undensitised inputs of the recovery problem at one cell.
template <class S>
struct C2P {
  S D, tau, S2, B2, BS, gamma;
};

// v^2 as a function of z from the momentum equation S_i = (z + B^2) v_i -
// (B.v) B_i with B.v = (B.S) / z.
template <class S>
S c2p_v2(const C2P<S>& in, const S& z) {
  const S zb = z + in.B2;
  return (in.S2 + in.BS * in.BS * (2.0 * z + in.B2) / (z * z)) / (zb * zb);
}

// Energy residual tau - tau(z); positive when z is too small.
template <class S>
S c2p_f(const C2P<S>& in, const S& z) {
  const S v2 = c2p_v2(in, z);
  const S iw = sqrt(S(1.0) - v2);           // 1/W
  const S press = (in.gamma - 1.0) / in.gamma * (z * iw * iw - in.D * iw);
  return in.tau + in.D - z - in.B2 + 0.5 * in.B2 * iw * iw + 0.5 * in.BS * in.BS / (z * z) + press;
}

// Reading R18: Newman-Hamlin fixed point over P from P0.  Returns true and
// (z, W) when |P_{k+1} - P_k| <= tol |P_{k+1}| within maxit iterations.
inline bool c2p_newman_hamlin(const C2P<double>& in, double P0, int maxit, double tol, double& z, double& W) {
  const double E = in.tau + in.D;
  double d = 0.5 * (in.B2 * in.S2 - in.BS * in.BS);
  if (d < 0.0) d = 0.0;  // Cauchy-Schwarz: negative only by round-off
  double P = P0;
  for (int it = 0; it < maxit; ++it) {
    const double a = E + P + 0.5 * in.B2;
    if (!(a > 0.0)) return false;
    const double r = 1.0 - 27.0 * d / (2.0 * a * a * a);
    if (!(r >= -1.0)) return false;  // d > 4 a^3 / 27: no root above 2a/3
    const double eps = a / 3.0 + (2.0 * a / 3.0) * std::cos(std::acos(std::min(r, 1.0)) / 3.0);
    const double zz = eps - in.B2;
    if (!(zz > 0.0)) return false;
    const double v2 = c2p_v2(in, zz);
    if (!(v2 < 1.0)) return false;
    const double iw = std::sqrt(1.0 - v2);
    const double Pn = (in.gamma - 1.0) / in.gamma * (zz * iw * iw - in.D * iw);
    const bool done = std::fabs(Pn - P) <= tol * std::fabs(Pn);
    P = Pn;
    if (done) {
      z = zz;
      W = 1.0 / iw;
      return std::isfinite(z) && std::isfinite(W);
    }
  }
  return false;
}

// Reading R20: recovery under the polytrope P = K rho^Gamma.  With
// rho = D / W, h = 1 + Gamma/(Gamma-1) K rho^(Gamma-1) and z = rho h W^2,
// the momentum equation g(W) = (z + B^2)^2 (1 - 1/W^2)
// - (B.S)^2 (2z + B^2) / z^2 - S^2 is <= 0 at W = 1 and grows without
// bound; its root W >= 1 is found by bisection (the upper end doubled until
// g > 0), to a relative width of 1e-15.  tau is not used.
template <class S, class Atm>
int con2prim_polytrope(const C2P<S>& in, const Spacetime<double>& st, const double gu3[3][3], const S Sl[3],
                       const S B[3], const Par<S>& p, S out[8], Atm atmosphere) {
  const double D = val(in.D), S2 = val(in.S2), B2 = val(in.B2), BS = val(in.BS);
  const double G = val(p.gamma), K = p.poly_K;
  if (!(D > 0.0)) return atmosphere();
  auto z_of = [&](double W) {
    const double rho = D / W;
    const double h = 1.0 + G / (G - 1.0) * K * std::pow(rho, G - 1.0);
    return rho * h * W * W;
  };
  auto g_of = [&](double W) {
    const double z = z_of(W);
    return (z + B2) * (z + B2) * (1.0 - 1.0 / (W * W)) - BS * BS * (2.0 * z + B2) / (z * z) - S2;
  };
  double lo = 1.0, hi = 2.0;
  int guard = 0;
  while (!(g_of(hi) > 0.0) && guard < 200) {
    lo = hi;
    hi *= 2.0;
    ++guard;
  }
  if (guard >= 200) return atmosphere();
  for (int it = 0; it < 400 && hi - lo > 1e-15 * hi; ++it) {
    const double m = 0.5 * (lo + hi);
    if (g_of(m) > 0.0) hi = m; else lo = m;
  }
  const double W = 0.5 * (lo + hi);
  const double z = z_of(W);
  const double rho = D / W;
  if (!(rho >= p.rho_atm) || !std::isfinite(z)) return atmosphere();
  // v_i = (S_i + (B.S / z) B_i) / (z + B^2), B_i = gamma_ij B^j
  double vl[3];
  for (int i = 0; i < 3; ++i) {
    double Bl = 0.0;
    for (int j = 0; j < 3; ++j) Bl += st.gam[i][j] * val(B[j]);
    vl[i] = (val(Sl[i]) + BS / z * Bl) / (z + B2);
  }
  out[0] = S(rho);
  for (int i = 0; i < 3; ++i) {
    double t = 0.0;
    for (int j = 0; j < 3; ++j) t += gu3[i][j] * vl[j];
    out[1 + i] = S(t);
  }
  out[4] = S(K * std::pow(rho, G));
  for (int i = 0; i < 3; ++i) out[5 + i] = B[i];
  return 0;
}

// Returns status 0 on success, 1 if the atmosphere was imposed, 2 if the
// pressure floor was applied.
template <class S>
int con2prim_cell(const S U[8], const double adm[10], const Par<S>& p, S out[8]) {
  Spacetime<double> st;
  spacetime_from_adm(adm, st);
  double gu3[3][3];
  invert_gj<double, 3>(st.gam, gu3);
  const double sg = st.sqrtgam;
  C2P<S> in;
  in.gamma = p.gamma;
  in.D = U[0] / sg;
  in.tau = U[4] / sg;
  S Sl[3], B[3];
  for (int i = 0; i < 3; ++i) { Sl[i] = U[1 + i] / sg; B[i] = U[5 + i] / sg; }
  in.S2 = S(0.0); in.B2 = S(0.0); in.BS = S(0.0);
  for (int i = 0; i < 3; ++i) {
    in.BS += B[i] * Sl[i];
    for (int j = 0; j < 3; ++j) {
      in.S2 += gu3[i][j] * Sl[i] * Sl[j];
      in.B2 += st.gam[i][j] * B[i] * B[j];
    }
  }
  auto atmosphere = [&]() {
    out[0] = S(p.rho_atm);
    for (int i = 0; i < 3; ++i) out[1 + i] = S(0.0);
    out[4] = S(p.p_atm);
    for (int i = 0; i < 3; ++i) out[5 + i] = B[i];
    return 1;
  };
  if (p.eos == EOS_POLYTROPE) return con2prim_polytrope(in, st, gu3, Sl, B, p, out, atmosphere);
  if (!(val(in.D) > 0.0) || !(val(in.tau) + val(in.D) > 0.0)) return atmosphere();
  // Value-level bisection bracket: sign(z) = +1 where v^2 >= 1 or f > 0;
  // lo_energy records whether the current lower end is positive through the
  // energy residual itself (v^2 < 1, f > 0) rather than through v^2 >= 1.
  C2P<double> iv;
  iv.D = val(in.D); iv.tau = val(in.tau); iv.S2 = val(in.S2); iv.B2 = val(in.B2);
  iv.BS = val(in.BS); iv.gamma = val(in.gamma);
  auto sign_class = [&](double z) {  // 0: f <= 0 inside v < 1; 1: f > 0 inside; 2: v^2 >= 1
    const double v2 = c2p_v2(iv, z);
    if (!(v2 < 1.0)) return 2;
    return c2p_f(iv, z) > 0.0 ? 1 : 0;
  };
  double zlo = 0.0;
  bool lo_energy = false;
  double zhi = 2.0 * iv.gamma * (iv.tau + iv.D) + iv.B2 + 1e-300;
  int guard = 0;
  for (int c = sign_class(zhi); c != 0 && guard < 200; c = sign_class(zhi)) {
    zlo = zhi;
    lo_energy = c == 1;
    zhi *= 2.0;
    ++guard;
  }
  if (guard >= 200) return atmosphere();
  for (int it = 0; it < 400; ++it) {
    const double zm = 0.5 * (zlo + zhi);
    const int c = sign_class(zm);
    if (c != 0) { zlo = zm; lo_energy = c == 1; } else { zhi = zm; }
    if (zhi - zlo <= 1e-15 * zhi) break;
  }
  // reading R12: no sign change of f inside v < 1 means no root
  if (!lo_energy) return atmosphere();
  const double zv = 0.5 * (zlo + zhi);
  // One Newton polish, carrying the derivative of the root with respect to
  // the inputs (implicit function theorem) when S is a dual number.
  Dual<1> zd(zv);
  zd.d[0] = 1.0;
  C2P<Dual<1>> i1;
  i1.D = iv.D; i1.tau = iv.tau; i1.S2 = iv.S2; i1.B2 = iv.B2; i1.BS = iv.BS; i1.gamma = iv.gamma;
  const double fz = c2p_f(i1, zd).d[0];
  S z = S(zv);
  if (std::isfinite(fz) && fz != 0.0) {
    const S corr = c2p_f(in, S(zv)) / fz;
    if (std::fabs(val(corr)) < 1e-6 * zv) z = S(zv) - corr;
  }
  const S v2 = c2p_v2(in, z);
  const S iw = sqrt(S(1.0) - v2);
  const S rho = in.D * iw;
  const S press = (in.gamma - 1.0) / in.gamma * (z * iw * iw - rho);
  if (!(val(rho) >= p.rho_atm) || !(val(v2) < 1.0) || !std::isfinite(val(press))) return atmosphere();
  int status = 0;
  S pout = press;
  if (!(val(press) > 0.0)) { pout = S(p.p_atm); status = 2; }  // reading R12: pressure floor
  S vl[3];
  // v_i = (S_i + (B.S / z) B_i) / (z + B^2) with B_i = gamma_ij B^j
  for (int i = 0; i < 3; ++i) {
    S Bl = S(0.0);
    for (int j = 0; j < 3; ++j) Bl += st.gam[i][j] * B[j];
    vl[i] = (Sl[i] + in.BS / z * Bl) / (z + in.B2);
  }
  out[0] = rho;
  for (int i = 0; i < 3; ++i) {
    S t = S(0.0);
    for (int j = 0; j < 3; ++j) t += gu3[i][j] * vl[j];
    out[1 + i] = t;
  }
  out[4] = pout;
  for (int i = 0; i < 3; ++i) out[5 + i] = B[i];
  return status;
}

template <class S>
int con2prim_block(const Grid& G, const Par<S>& p, const S* cons, const double* metric, S* prim, int8_t* status) {
  int nfail = 0;
  const int g = G.ng;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nfail)
  for (int k = g; k < g + G.n[2]; ++k)
    for (int j = g; j < g + G.n[1]; ++j)
      for (int i = g; i < g + G.n[0]; ++i) {
        const long c = G.at(i, j, k);
        double adm[10];
        load_adm(G, metric, c, adm);
        S U[8], P[8];
        for (int q = 0; q < 8; ++q) U[q] = cons[q * G.ncell + c];
        const int st = con2prim_cell(U, adm, p, P);
        for (int q = 0; q < 8; ++q) prim[q * G.ncell + c] = P[q];
        if (status) status[c] = (int8_t)st;
        nfail += (st != 0);
      }
  return nfail;
}

// ------------------------------------------------------- ghost zones (R9) --
template <class S>
void fill_ghosts_block(const Grid& G, int bc, int nvar, S* a) {
  const int g = G.ng;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < G.N[2]; ++k)
    for (int j = 0; j < G.N[1]; ++j)
      for (int i = 0; i < G.N[0]; ++i) {
        if (G.interior(i, j, k)) continue;
        int c[3] = {i, j, k}, s[3];
        for (int d = 0; d < 3; ++d) {
          if (bc == BC_PERIODIC) {
            int r = (c[d] - g) % G.n[d];
            if (r < 0) r += G.n[d];
            s[d] = g + r;
          } else {
            s[d] = std::min(std::max(c[d], g), g + G.n[d] - 1);
          }
        }
        const long dst = G.at(i, j, k), src = G.at(s[0], s[1], s[2]);
        for (int q = 0; q < nvar; ++q) a[q * G.ncell + dst] = a[q * G.ncell + src];
      }
}

// -------------------------------------------------- time integration (R10) --
// One step; on entry prim is consistent with cons (ghosts filled); on exit
// cons holds U^{n+1} and prim its primitives (ghosts filled).
template <class S>
int rk_step_block(const Grid& G, const Par<S>& p, int scheme, double dt, S* cons, S* prim,
                  const double* metric, const double* Kij, int8_t* status) {
  const long n8 = 8 * G.ncell;
  std::vector<S> U0(cons, cons + n8), L(n8), acc;
  int nfail = 0;
  auto interior_update = [&](auto fn) {
    for (int k = G.ng; k < G.ng + G.n[2]; ++k)
      for (int j = G.ng; j < G.ng + G.n[1]; ++j)
        for (int i = G.ng; i < G.ng + G.n[0]; ++i) {
          const long c = G.at(i, j, k);
          for (int q = 0; q < 8; ++q) fn(q * G.ncell + c);
        }
  };
  auto recover = [&]() {
    nfail += con2prim_block(G, p, cons, metric, prim, status);
    fill_ghosts_block(G, p.bc, 8, prim);
  };
  if (scheme == RK2) {
    rhs_block(G, p, prim, metric, Kij, L.data());
    interior_update([&](long x) { cons[x] = U0[x] + dt * L[x]; });
    recover();
    rhs_block(G, p, prim, metric, Kij, L.data());
    interior_update([&](long x) { cons[x] = 0.5 * U0[x] + 0.5 * (cons[x] + dt * L[x]); });
    recover();
  } else if (scheme == RK3) {
    rhs_block(G, p, prim, metric, Kij, L.data());
    interior_update([&](long x) { cons[x] = U0[x] + dt * L[x]; });
    recover();
    rhs_block(G, p, prim, metric, Kij, L.data());
    interior_update([&](long x) { cons[x] = 0.75 * U0[x] + 0.25 * (cons[x] + dt * L[x]); });
    recover();
    rhs_block(G, p, prim, metric, Kij, L.data());
    interior_update([&](long x) { cons[x] = (1.0 / 3.0) * U0[x] + (2.0 / 3.0) * (cons[x] + dt * L[x]); });
    recover();
  } else {  // classical RK4
    acc.assign(n8, S(0.0));
    const double cstage[3] = {0.5, 0.5, 1.0};
    const double wstage[4] = {1.0, 2.0, 2.0, 1.0};
    for (int s = 0; s < 4; ++s) {
      rhs_block(G, p, prim, metric, Kij, L.data());
      if (s < 3) {
        interior_update([&](long x) {
          acc[x] = acc[x] + wstage[s] * L[x];
          cons[x] = U0[x] + (cstage[s] * dt) * L[x];
        });
      } else {
        interior_update([&](long x) { cons[x] = U0[x] + (dt / 6.0) * (acc[x] + L[x]); });
      }
      recover();
    }
  }
  return nfail;
}

// ---------------------------------------- constrained transport (R19) --
// Face field bface[a * ncell + idx]: component a on the lower a-face of
// cell idx (array indices, ghosts included); the interior faces have
// a-index ng .. ng + n_a and interior transverse indices.

// Rate of change of the face field: -curl E on every interior face.
template <class S>
void ct_rate(const Grid& G, const Par<S>& p, const S* prim, const double* metric, S* dbdt) {
  const int g = G.ng;
  const long st[3] = {1, G.N[0], (long)G.N[0] * G.N[1]};
  // face fluxes of the field components: Fb[(3 d + comp) * ncell + idx] = F_d(B^comp) on the lower
  // d-face of cell idx, for d-index g .. g + n_d and transverse indices g - 1 .. g + n
  std::vector<S> Fb((size_t)9 * G.ncell, S(0.0));
  for (int d = 0; d < 3; ++d) {
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      lo[e] = e == d ? g : g - 1;
      hi[e] = g + G.n[e];
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          S F[8];
          face_flux(G, p, prim, metric, d, i, j, k, F);
          for (int c = 0; c < 3; ++c) Fb[(3 * d + c) * G.ncell + G.at(i, j, k)] = F[5 + c];
        }
  }
  // edge fields: E[c * ncell + idx] on the c-edge at the corner of cell idx that is lower in a and b,
  // (c, a, b) cyclic: E_c = (-F_a(B^b)[idx - e_b] - F_a(B^b)[idx] + F_b(B^a)[idx - e_a] + F_b(B^a)[idx]) / 4
  std::vector<S> E((size_t)3 * G.ncell, S(0.0));
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    for (int k = g; k <= g + G.n[2]; ++k)
      for (int j = g; j <= g + G.n[1]; ++j)
        for (int i = g; i <= g + G.n[0]; ++i) {
          const long x = G.at(i, j, k);
          const S* Fab = Fb.data() + (3 * a + b) * G.ncell;
          const S* Fba = Fb.data() + (3 * b + a) * G.ncell;
          E[c * G.ncell + x] = 0.25 * (-Fab[x - st[b]] - Fab[x] + Fba[x - st[a]] + Fba[x]);
        }
  }
  // d B^a / dt = -(E_c[idx + e_b] - E_c[idx]) / dx_b + (E_b[idx + e_c] - E_b[idx]) / dx_c, (a, b, c) cyclic
  for (long x = 0; x < 3 * G.ncell; ++x) dbdt[x] = S(0.0);
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    int hi[3] = {g + G.n[0] - 1, g + G.n[1] - 1, g + G.n[2] - 1};
    hi[a] = g + G.n[a];
    for (int k = g; k <= hi[2]; ++k)
      for (int j = g; j <= hi[1]; ++j)
        for (int i = g; i <= hi[0]; ++i) {
          const long x = G.at(i, j, k);
          const S* Ec = E.data() + c * G.ncell;
          const S* Eb = E.data() + b * G.ncell;
          dbdt[a * G.ncell + x] = -(Ec[x + st[b]] - Ec[x]) / G.dx[b] + (Eb[x + st[c]] - Eb[x]) / G.dx[c];
        }
  }
}

// Cell-centred densitised field of the interior cells := mean of the two faces.
template <class S>
void ct_face_to_cell(const Grid& G, const S* bface, S* cons) {
  const long st[3] = {1, G.N[0], (long)G.N[0] * G.N[1]};
  for (int k = G.ng; k < G.ng + G.n[2]; ++k)
    for (int j = G.ng; j < G.ng + G.n[1]; ++j)
      for (int i = G.ng; i < G.ng + G.n[0]; ++i) {
        const long x = G.at(i, j, k);
        for (int a = 0; a < 3; ++a)
          cons[(5 + a) * G.ncell + x] = 0.5 * (bface[a * G.ncell + x] + bface[a * G.ncell + x + st[a]]);
      }
}

// Discrete divergence of the face field on the interior cells.
template <class S>
void ct_divergence(const Grid& G, const S* bface, S* div) {
  const long st[3] = {1, G.N[0], (long)G.N[0] * G.N[1]};
  for (long x = 0; x < G.ncell; ++x) div[x] = S(0.0);
  for (int k = G.ng; k < G.ng + G.n[2]; ++k)
    for (int j = G.ng; j < G.ng + G.n[1]; ++j)
      for (int i = G.ng; i < G.ng + G.n[0]; ++i) {
        const long x = G.at(i, j, k);
        S dv = S(0.0);
        for (int a = 0; a < 3; ++a) dv = dv + (bface[a * G.ncell + x + st[a]] - bface[a * G.ncell + x]) / G.dx[a];
        div[x] = dv;
      }
}

// One SSP-RK2 / SSP-RK3 / RK4 step with constrained transport: the fluid
// variables as in rk_step_block, the face field by the same stage formulas
// with ct_rate, the cell field taken from the faces before every recovery.
template <class S>
int ct_rk_step_block(const Grid& G, const Par<S>& p, int scheme, double dt, S* cons, S* prim, S* bface,
                     const double* metric) {
  const long n8 = 8 * G.ncell, n3 = 3 * G.ncell;
  std::vector<S> U0(cons, cons + n8), L(n8), acc(n8, S(0.0));
  std::vector<S> B0(bface, bface + n3), dB(n3), accB(n3, S(0.0));
  int nfail = 0;
  const int nstage = scheme == RK2 ? 2 : (scheme == RK3 ? 3 : 4);
  auto update = [&](S* u, const S* u0, const S* l, S* ac, long x, int s) {
    if (scheme == RK2) {
      u[x] = s == 0 ? u0[x] + dt * l[x] : 0.5 * u0[x] + 0.5 * (u[x] + dt * l[x]);
    } else if (scheme == RK3) {
      if (s == 0) u[x] = u0[x] + dt * l[x];
      else if (s == 1) u[x] = 0.75 * u0[x] + 0.25 * (u[x] + dt * l[x]);
      else u[x] = (1.0 / 3.0) * u0[x] + (2.0 / 3.0) * (u[x] + dt * l[x]);
    } else {
      const double cst[3] = {0.5, 0.5, 1.0}, wst[3] = {1.0, 2.0, 2.0};
      if (s < 3) {
        ac[x] = ac[x] + wst[s] * l[x];
        u[x] = u0[x] + (cst[s] * dt) * l[x];
      } else {
        u[x] = u0[x] + (dt / 6.0) * (ac[x] + l[x]);
      }
    }
  };
  for (int s = 0; s < nstage; ++s) {
    rhs_block(G, p, prim, metric, nullptr, L.data());
    ct_rate(G, p, prim, metric, dB.data());
    for (int k = G.ng; k < G.ng + G.n[2]; ++k)
      for (int j = G.ng; j < G.ng + G.n[1]; ++j)
        for (int i = G.ng; i < G.ng + G.n[0]; ++i)
          for (int q = 0; q < 5; ++q) update(cons, U0.data(), L.data(), acc.data(), q * G.ncell + G.at(i, j, k), s);
    for (int a = 0; a < 3; ++a) {
      int hi[3] = {G.ng + G.n[0] - 1, G.ng + G.n[1] - 1, G.ng + G.n[2] - 1};
      hi[a] = G.ng + G.n[a];
      for (int k = G.ng; k <= hi[2]; ++k)
        for (int j = G.ng; j <= hi[1]; ++j)
          for (int i = G.ng; i <= hi[0]; ++i) update(bface, B0.data(), dB.data(), accB.data(), a * G.ncell + G.at(i, j, k), s);
    }
    ct_face_to_cell(G, (const S*)bface, cons);
    nfail += con2prim_block(G, p, cons, metric, prim, (int8_t*)nullptr);
    fill_ghosts_block(G, p.bc, 8, prim);
  }
  return nfail;
}

// --------------------------------------------- two-level AMR (R14-R17) --
// A fine block at placement lo: its interior cell i (0-based, ghosts i < 0
// or i >= n) lies in the coarse interior cell lo + floor(i / 2) along each
// axis, and its spacing is half the coarse one.
inline int floor_half(int i) { return i >= 0 ? i / 2 : -((1 - i) / 2); }

// R14: covered coarse cells of `coarse` := mean of their 8 fine children.
template <class S>
void restrict_block(const Grid& C, S* coarse, const Grid& F, const S* fine, const int lo[3], int nvar) {
  for (int K = 0; K < F.n[2] / 2; ++K)
    for (int J = 0; J < F.n[1] / 2; ++J)
      for (int I = 0; I < F.n[0] / 2; ++I)
        for (int q = 0; q < nvar; ++q) {
          S sum = S(0.0);
          for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
              for (int a = 0; a < 2; ++a)
                sum = sum + fine[q * F.ncell + F.at(F.ng + 2 * I + a, F.ng + 2 * J + b, F.ng + 2 * K + c)];
          coarse[q * C.ncell + C.at(C.ng + lo[0] + I, C.ng + lo[1] + J, C.ng + lo[2] + K)] = sum / 8.0;
        }
}

// R15: fine points (all, or the ghosts only) from the coarse parents.
template <class S>
void prolongate_block(const Grid& C, const S* coarse, const Grid& F, S* fine, const int lo[3], int nvar,
                      bool ghosts_only) {
  for (int k = -F.ng; k < F.n[2] + F.ng; ++k)
    for (int j = -F.ng; j < F.n[1] + F.ng; ++j)
      for (int i = -F.ng; i < F.n[0] + F.ng; ++i) {
        const bool inside = i >= 0 && i < F.n[0] && j >= 0 && j < F.n[1] && k >= 0 && k < F.n[2];
        if (ghosts_only && inside) continue;
        const int fi[3] = {i, j, k};
        int P[3];
        double off[3];
        for (int d = 0; d < 3; ++d) {
          P[d] = C.ng + lo[d] + floor_half(fi[d]);
          off[d] = (fi[d] - 2 * floor_half(fi[d]) == 0) ? -0.25 : 0.25;
        }
        for (int q = 0; q < nvar; ++q) {
          const S* u = coarse + q * C.ncell;
          const S u0 = u[C.at(P[0], P[1], P[2])];
          S val = u0;
          for (int d = 0; d < 3; ++d) {
            int m[3] = {P[0], P[1], P[2]}, pl[3] = {P[0], P[1], P[2]};
            m[d] -= 1;
            pl[d] += 1;
            const S slope = minmod(u0 - u[C.at(m[0], m[1], m[2])], u[C.at(pl[0], pl[1], pl[2])] - u0);
            val = val + off[d] * slope;
          }
          fine[q * F.ncell + F.at(F.ng + i, F.ng + j, F.ng + k)] = val;
        }
      }
}

// R16: adds scale * (change of the coarse RHS) to `out` for the uncovered
// coarse cells next to the fine block, the coarse interface flux being
// replaced by the mean of its 4 fine face fluxes.
template <class S>
void reflux_block(const Grid& C, const Par<S>& p, const S* cprim, const double* cmetric, const Grid& F,
                  const S* fprim, const double* fmetric, const int lo[3], double scale, S* out) {
  const int nc[3] = {F.n[0] / 2, F.n[1] / 2, F.n[2] / 2};
  for (int d = 0; d < 3; ++d) {
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    for (int side = 0; side < 2; ++side)
      for (int B = 0; B < nc[b]; ++B)
        for (int A = 0; A < nc[a]; ++A) {
          int Ic[3];
          Ic[d] = lo[d] + (side ? nc[d] : 0);
          Ic[a] = lo[a] + A;
          Ic[b] = lo[b] + B;
          S Fc[8];
          face_flux(C, p, cprim, cmetric, d, C.ng + Ic[0], C.ng + Ic[1], C.ng + Ic[2], Fc);
          S Ff[8];
          for (int q = 0; q < 8; ++q) Ff[q] = S(0.0);
          for (int ib = 0; ib < 2; ++ib)
            for (int ia = 0; ia < 2; ++ia) {
              int If[3];
              If[d] = side ? F.n[d] : 0;
              If[a] = 2 * A + ia;
              If[b] = 2 * B + ib;
              S Fx[8];
              face_flux(F, p, fprim, fmetric, d, F.ng + If[0], F.ng + If[1], F.ng + If[2], Fx);
              for (int q = 0; q < 8; ++q) Ff[q] = Ff[q] + Fx[q];
            }
          int Icell[3] = {Ic[0], Ic[1], Ic[2]};
          if (!side) Icell[d] -= 1;                  // the face is this cell's upper face
          const double sign = side ? 1.0 : -1.0;     // ... or its lower face
          const long cc = C.at(C.ng + Icell[0], C.ng + Icell[1], C.ng + Icell[2]);
          for (int q = 0; q < 8; ++q) out[q * C.ncell + cc] = out[q * C.ncell + cc] + scale * sign * (0.25 * Ff[q] - Fc[q]) / C.dx[d];
        }
  }
}

// R17: one composite SSP-RK2 / SSP-RK3 / RK4 step of a coarse block and nf
// fine blocks.  Returns the number of failed recoveries.
template <class S>
int amr2_step(const Grid& C, const Par<S>& p, int scheme, double dt, S* ccons, S* cprim, const double* cmetric,
              int nf, const Grid* Fg, S* const* fcons, S* const* fprim, const double* const* fmetric,
              const int* lo) {
  const int nb = nf + 1;
  std::vector<const Grid*> G(nb);
  std::vector<S*> U(nb), P(nb);
  std::vector<const double*> M(nb);
  G[0] = &C; U[0] = ccons; P[0] = cprim; M[0] = cmetric;
  for (int f = 0; f < nf; ++f) { G[f + 1] = &Fg[f]; U[f + 1] = fcons[f]; P[f + 1] = fprim[f]; M[f + 1] = fmetric[f]; }
  std::vector<std::vector<S>> U0(nb), L(nb), acc(nb);
  for (int b = 0; b < nb; ++b) {
    const long n8 = 8 * G[b]->ncell;
    U0[b].assign(U[b], U[b] + n8);
    L[b].assign(n8, S(0.0));
    acc[b].assign(n8, S(0.0));
  }
  int nfail = 0;
  const int nstage = scheme == RK2 ? 2 : (scheme == RK3 ? 3 : 4);
  for (int s = 0; s < nstage; ++s) {
    for (int b = 0; b < nb; ++b) rhs_block(*G[b], p, P[b], M[b], nullptr, L[b].data());
    for (int f = 0; f < nf; ++f) reflux_block(C, p, cprim, cmetric, Fg[f], P[f + 1], M[f + 1], lo + 3 * f, 1.0, L[0].data());
    for (int b = 0; b < nb; ++b) {
      const Grid& g = *G[b];
      for (int k = g.ng; k < g.ng + g.n[2]; ++k)
        for (int j = g.ng; j < g.ng + g.n[1]; ++j)
          for (int i = g.ng; i < g.ng + g.n[0]; ++i)
            for (int q = 0; q < 8; ++q) {
              const long x = q * g.ncell + g.at(i, j, k);
              S* u = U[b];
              const S* u0 = U0[b].data();
              const S l = L[b][x];
              if (scheme == RK2) {
                u[x] = s == 0 ? u0[x] + dt * l : 0.5 * u0[x] + 0.5 * (u[x] + dt * l);
              } else if (scheme == RK3) {
                if (s == 0) u[x] = u0[x] + dt * l;
                else if (s == 1) u[x] = 0.75 * u0[x] + 0.25 * (u[x] + dt * l);
                else u[x] = (1.0 / 3.0) * u0[x] + (2.0 / 3.0) * (u[x] + dt * l);
              } else {
                const double cst[3] = {0.5, 0.5, 1.0}, wst[3] = {1.0, 2.0, 2.0};
                if (s < 3) {
                  acc[b][x] = acc[b][x] + wst[s] * l;
                  u[x] = u0[x] + (cst[s] * dt) * l;
                } else {
                  u[x] = u0[x] + (dt / 6.0) * (acc[b][x] + l);
                }
              }
            }
    }
    for (int f = 0; f < nf; ++f) restrict_block(C, ccons, Fg[f], fcons[f], lo + 3 * f, 8);
    for (int b = 0; b < nb; ++b) nfail += con2prim_block(*G[b], p, U[b], M[b], P[b], (int8_t*)nullptr);
    fill_ghosts_block(C, p.bc, 8, cprim);
    for (int f = 0; f < nf; ++f) prolongate_block(C, (const S*)cprim, Fg[f], fprim[f], lo + 3 * f, 8, true);
  }
  return nfail;
}

}  // namespace orc

// ======================================================================
// C entry points (double precision; one forward-mode entry point).
// Arrays are SoA [var][z][y][x] with x fastest, N = n + 2 ng per axis.
// ======================================================================
using namespace orc;

static Par<double> to_par(const OParams* q) {
  Par<double> p;
  p.gamma = q->gamma; p.recon = q->recon; p.bc = q->bc;
  p.rho_atm = q->rho_atm; p.p_atm = q->p_atm; p.weno_eps = q->weno_eps;
  p.eos = q->eos; p.poly_K = q->poly_K;
  // reading R20: the polytrope's atmosphere pressure
  if (p.eos == EOS_POLYTROPE) p.p_atm = q->poly_K * std::pow(q->rho_atm, q->gamma);
  return p;
}

extern "C" {

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void oracle_prim2con(const int* n3, int ng, const double* dx3, double gamma,
                     const double* prim, const double* metric, double* cons) {
  Grid G; G.init(n3, ng, dx3);
  prim2con_block<double>(G, gamma, prim, metric, cons);
}

// prim -> cons under the EOS of q (reading R20 for the polytrope).
void oracle_prim2con_eos(const int* n3, int ng, const double* dx3, const OParams* q, const double* prim,
                         const double* metric, double* cons) {
  Grid G; G.init(n3, ng, dx3);
  prim2con_block<double>(G, q->gamma, prim, metric, cons, q->eos, q->poly_K);
}

int oracle_con2prim(const int* n3, int ng, const double* dx3, const OParams* q,
                    const double* cons, const double* metric, double* prim, int8_t* status) {
  Grid G; G.init(n3, ng, dx3);
  return con2prim_block<double>(G, to_par(q), cons, metric, prim, status);
}

void oracle_fill_ghosts(const int* n3, int ng, int bc, int nvar, double* a) {
  const double dx[3] = {1, 1, 1};
  Grid G; G.init(n3, ng, dx);
  fill_ghosts_block<double>(G, bc, nvar, a);
}

void oracle_rhs(const int* n3, int ng, const double* dx3, const OParams* q, const double* prim,
                const double* metric, const double* Kij, double* rhs) {
  Grid G; G.init(n3, ng, dx3);
  rhs_block<double>(G, to_par(q), prim, metric, Kij, rhs);
}

void oracle_rhs_cells(const int* n3, int ng, const double* dx3, const OParams* q, const double* prim,
                      const double* metric, const double* Kij, long ncells, const int32_t* ijk, double* out) {
  Grid G; G.init(n3, ng, dx3);
  const Par<double> p = to_par(q);
#pragma omp parallel for schedule(dynamic, 16)
  for (long s = 0; s < ncells; ++s) {
    double r[8];
    rhs_one_cell(G, p, prim, metric, Kij, ijk[3 * s], ijk[3 * s + 1], ijk[3 * s + 2], r);
    for (int q2 = 0; q2 < 8; ++q2) out[8 * s + q2] = r[q2];
  }
}

// Eq. 13 source vector alone at selected cells.
void oracle_source_cells(const int* n3, int ng, const double* dx3, const OParams* q, const double* prim,
                         const double* metric, const double* Kij, long ncells, const int32_t* ijk, double* out) {
  Grid G; G.init(n3, ng, dx3);
  const Par<double> p = to_par(q);
  for (long s = 0; s < ncells; ++s) {
    double r[8];
    source_cell(G, p, prim, metric, Kij, ijk[3 * s], ijk[3 * s + 1], ijk[3 * s + 2], r);
    for (int q2 = 0; q2 < 8; ++q2) out[8 * s + q2] = r[q2];
  }
}

int oracle_rk_step(const int* n3, int ng, const double* dx3, const OParams* q, int scheme, double dt,
                   double* cons, double* prim, const double* metric, const double* Kij, int8_t* status) {
  Grid G; G.init(n3, ng, dx3);
  return rk_step_block<double>(G, to_par(q), scheme, dt, cons, prim, metric, Kij, status);
}

// Point-wise physics at one state: conserved vector, the three physical
// fluxes and the signal speeds.  adm may be NULL (Minkowski).
void oracle_point(const double* prim8, const double* adm10, double gamma, double* U8, double* F24, double* lam6,
                  double* extra4) {
  double adm[10];
  if (adm10) for (int q = 0; q < 10; ++q) adm[q] = adm10[q]; else flat_adm(adm);
  Spacetime<double> st;
  spacetime_from_adm(adm, st);
  Fluid<double> f;
  fluid_from_prim(prim8, st, gamma, f);
  conserved(f, st, U8);
  for (int d = 0; d < 3; ++d) {
    flux(f, st, d, F24 + 8 * d);
    wave_speeds(f, st, gamma, d, lam6[2 * d], lam6[2 * d + 1]);
  }
  if (extra4) {
    extra4[0] = f.W;
    extra4[1] = f.b2;
    double bu = 0.0;  // b^mu u_mu, zero by construction
    for (int m = 0; m < 4; ++m) bu += f.b[m] * f.ul[m];
    extra4[2] = bu;
    double uu = 0.0;  // u^mu u_mu = -1
    for (int m = 0; m < 4; ++m) uu += f.u[m] * f.ul[m];
    extra4[3] = uu;
  }
}

// HLLE flux between two primitive states at a face with metric adm10 (NULL = flat).
void oracle_hlle(const double* pL, const double* pR, const double* adm10, double gamma, int dir, double* F8,
                 double* speeds4) {
  double adm[10];
  if (adm10) for (int q = 0; q < 10; ++q) adm[q] = adm10[q]; else flat_adm(adm);
  FaceOut<double> fo;
  hlle(pL, pR, adm, gamma, dir, fo);
  for (int q = 0; q < 8; ++q) F8[q] = fo.F[q];
  if (speeds4) { speeds4[0] = fo.lmL; speeds4[1] = fo.lpL; speeds4[2] = fo.lmR; speeds4[3] = fo.lpR; }
}

// Face states of a 1D array u[0..n) for faces between cells c-1 and c,
// c = 3 .. n-3 (the six-point stencil must fit).  uL, uR have n entries;
// entries outside that range are left untouched.
void oracle_reconstruct_1d(int recon, double eps, int n, const double* u, double* uL, double* uR) {
  for (int c = 3; c <= n - 3; ++c) reconstruct_face(recon, eps, u + c - 3, uL[c], uR[c]);
}

// Con2prim of one cell; returns the status.
// Newman-Hamlin recovery of one flat-space state from the pressure guess P0
// (reading R18): returns 0 and prim8 on convergence, 1 otherwise.
int oracle_con2prim_nh_point(const double* U8, const OParams* q, double P0, double* prim8) {
  C2P<double> in;
  in.D = U8[0];
  in.tau = U8[4];
  in.S2 = U8[1] * U8[1] + U8[2] * U8[2] + U8[3] * U8[3];
  in.B2 = U8[5] * U8[5] + U8[6] * U8[6] + U8[7] * U8[7];
  in.BS = U8[5] * U8[1] + U8[6] * U8[2] + U8[7] * U8[3];
  in.gamma = q->gamma;
  double z = 0.0, W = 1.0;
  if (!c2p_newman_hamlin(in, P0, 10000, 1e-15, z, W)) return 1;
  const double rho = in.D / W;
  prim8[0] = rho;
  for (int i = 0; i < 3; ++i) prim8[1 + i] = (U8[1 + i] + in.BS / z * U8[5 + i]) / (z + in.B2);
  prim8[4] = (in.gamma - 1.0) / in.gamma * (z / (W * W) - rho);
  for (int i = 0; i < 3; ++i) prim8[5 + i] = U8[5 + i];
  return 0;
}

int oracle_con2prim_point(const double* U8, const double* adm10, const OParams* q, double* prim8) {
  double adm[10];
  if (adm10) for (int k = 0; k < 10; ++k) adm[k] = adm10[k]; else flat_adm(adm);
  return con2prim_cell<double>(U8, adm, to_par(q), prim8);
}

// Forward-mode directional derivative of the end-state functional
//   L = sum_interior rho^2 dV   (sqrt(gamma) dV in curved space)
// after nsteps steps, starting from interior primitives prim0 (full array,
// ghosts ignored and refilled) perturbed along dprim0 and Gamma along dgamma.
// Returns the number of failed recoveries; *L and *dL receive value and derivative.
int oracle_loss_jvp(const int* n3, int ng, const double* dx3, const OParams* q, int scheme, double dt, int nsteps,
                    const double* prim0, const double* dprim0, double dgamma, const double* metric,
                    const double* Kij, double* L, double* dL) {
  typedef Dual<1> D1;
  Grid G; G.init(n3, ng, dx3);
  Par<D1> p;
  p.gamma = D1(q->gamma); p.gamma.d[0] = dgamma;
  p.recon = q->recon; p.bc = q->bc; p.rho_atm = q->rho_atm; p.p_atm = q->p_atm; p.weno_eps = q->weno_eps;
  const long n8 = 8 * G.ncell;
  std::vector<D1> prim(n8), cons(n8);
  for (long x = 0; x < n8; ++x) { prim[x] = D1(prim0[x]); prim[x].d[0] = dprim0 ? dprim0[x] : 0.0; }
  fill_ghosts_block(G, p.bc, 8, prim.data());
  prim2con_block(G, p.gamma, prim.data(), metric, cons.data());
  int nfail = 0;
  for (int s = 0; s < nsteps; ++s)
    nfail += rk_step_block(G, p, scheme, dt, cons.data(), prim.data(), metric, Kij, (int8_t*)nullptr);
  D1 acc(0.0);
  const double dV = G.dx[0] * G.dx[1] * G.dx[2];
  for (int k = G.ng; k < G.ng + G.n[2]; ++k)
    for (int j = G.ng; j < G.ng + G.n[1]; ++j)
      for (int i = G.ng; i < G.ng + G.n[0]; ++i) {
        const long c = G.at(i, j, k);
        double sg = 1.0;
        if (metric) {
          double adm[10];
          for (int qq = 0; qq < 10; ++qq) adm[qq] = metric[qq * G.ncell + c];
          Spacetime<double> st;
          spacetime_from_adm(adm, st);
          sg = st.sqrtgam;
        }
        acc += (sg * dV) * (prim[c] * prim[c]);
      }
  *L = acc.v;
  *dL = acc.d[0];
  return nfail;
}

// Constrained transport (R19).  bface: 3 x ncell face field (see ct_rate).
void oracle_ct_rate(const int* n3, int ng, const double* dx3, const OParams* q, const double* prim,
                    const double* metric, double* dbdt) {
  Grid G; G.init(n3, ng, dx3);
  ct_rate<double>(G, to_par(q), prim, metric, dbdt);
}

void oracle_ct_divergence(const int* n3, int ng, const double* dx3, const double* bface, double* div) {
  Grid G; G.init(n3, ng, dx3);
  ct_divergence<double>(G, bface, div);
}

int oracle_ct_rk_step(const int* n3, int ng, const double* dx3, const OParams* q, int scheme, double dt,
                      double* cons, double* prim, double* bface, const double* metric) {
  Grid G; G.init(n3, ng, dx3);
  return ct_rk_step_block<double>(G, to_par(q), scheme, dt, cons, prim, bface, metric);
}

// Two-level AMR transfer (R14-R17).  Fine grids carry placements lo[3].
void oracle_restrict(const int* cn, int cng, const double* cdx, double* coarse, const int* fn, int fng,
                     const double* fdx, const double* fine, const int* lo, int nvar) {
  Grid C; C.init(cn, cng, cdx);
  Grid F; F.init(fn, fng, fdx);
  restrict_block<double>(C, coarse, F, fine, lo, nvar);
}

void oracle_prolongate(const int* cn, int cng, const double* cdx, const double* coarse, const int* fn, int fng,
                       const double* fdx, double* fine, const int* lo, int nvar, int ghosts_only) {
  Grid C; C.init(cn, cng, cdx);
  Grid F; F.init(fn, fng, fdx);
  prolongate_block<double>(C, coarse, F, fine, lo, nvar, ghosts_only != 0);
}

void oracle_reflux(const int* cn, int cng, const double* cdx, const OParams* q, const double* cprim,
                   const double* cmetric, const int* fn, int fng, const double* fdx, const double* fprim,
                   const double* fmetric, const int* lo, double scale, double* out) {
  Grid C; C.init(cn, cng, cdx);
  Grid F; F.init(fn, fng, fdx);
  reflux_block<double>(C, to_par(q), cprim, cmetric, F, fprim, fmetric, lo, scale, out);
}

// fine blocks: nf of them; fn, fdx, lo are 3 * nf arrays; fcons, fprim,
// fmetric arrays of nf pointers (fmetric entries may be NULL).
int oracle_amr2_step(const int* cn, int ng, const double* cdx, const OParams* q, int scheme, double dt,
                     double* ccons, double* cprim, const double* cmetric, int nf, const int* fn, const double* fdx,
                     double* const* fcons, double* const* fprim, const double* const* fmetric, const int* lo) {
  Grid C; C.init(cn, ng, cdx);
  std::vector<Grid> F(nf);
  for (int f = 0; f < nf; ++f) F[f].init(fn + 3 * f, ng, fdx + 3 * f);
  return amr2_step<double>(C, to_par(q), scheme, dt, ccons, cprim, cmetric, nf, F.data(), fcons, fprim, fmetric, lo);
}

}  // extern "C"
