// Pair interactions of the centroid-collocation boundary integral operator.
//
// For a target element i (centroid x_i, unit normal n_i) and a source element
// j (centroid x_j, unit normal n_j, area ds_j), with d = x_i - x_j, r = |d|,
// s = 1/r, e = exp(-kappa r), t = e (1 + kappa r),
// w = e (3 + 3 kappa r + kappa^2 r^2), c_i = n_i.d, c_j = n_j.d,
// c_ij = n_i.n_j and eps = eps_out / eps_in, the four kernels of Sec. 2.2.1
// (Eqs. for K1-K4, with the normal derivative in x taken as +n_x.grad_x)
// are, times 4 pi:
//   K1 = (1 - e) s                      K2 = (eps t - 1) c_j s^3
//   K3 = (t / eps - 1) c_i s^3          K4 = (t - 1) c_ij s^3 - (w - 3) c_i c_j s^5
// The mat-vec of Eqs. 5-6 needs, per pair,
//   K1 ds_j psi_j + K2 ds_j phi_j   and   K3 ds_j psi_j + K4 ds_j phi_j.
// Folding the source's area and values into its record,
//   a_j = ds_j psi_j,   m_j = ds_j phi_j n_j,
// these become
//   P = s [ (1 - e) a_j + (eps t - 1) (m_j.d) s^2 ]
//   Q = s^3 [ (t/eps - 1) c_i a_j + (t - 1) (n_i.m_j) - (w - 3) c_i (m_j.d) s^2 ]
// and w - 3 = 3 (t - 1) + (t - e) kappa r.  The 1/(4 pi) and the minus sign
// are applied once per output in the reduction kernel.
//
// The self pair j = i, omitted in Eqs. 5-6, is removed by setting s = 0 for
// it (the callers pass `self` only for source tiles that overlap the thread's
// own targets, so the common path carries no mask).  Every other factor is
// finite there, so both sums receive an exact zero.  Padding records carry
// zero values and m = 0 at a far-away position, and also add exact zeros.
// 1/r is clamped to S_MAX so that absurd inputs (distinct centroids closer
// than 1e-6 A) stay finite; such inputs are rejected at surface creation.
#pragma once
#include <cuda_runtime.h>

namespace bipb {

constexpr float kSMaxF = 1.0e6f;   // 1/r clamp: pairs closer than 1e-6 A act as self pairs
constexpr double kSMaxD = 1.0e6;
constexpr double kPi = 3.14159265358979323846;
constexpr double kCoulomb = 332.0716;           // Sec. 2.1: phi * 332.0716 -> kcal/mol/e
constexpr double kKcal = 4.0 * kPi * 332.0716;  // internal units (G0 carries 1/(4 pi)) -> kcal

template <typename T>
struct PairConst {
  T eps;     // eps_out / eps_in
  T inveps;  // 1 / eps
  T kappa;   // inverse Debye length
  T nkl2e;   // -kappa * log2(e), the ex2 argument scale (FP32 path)
};

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/r (clamped; 0 for the self pair) and exp(-kappa r) for both precisions.
template <bool MASK>
__device__ __forceinline__ void radial(float r2, bool self, const PairConst<float>& c, float& s,
                                       float& r, float& e) {
  s = fminf(rsqrt_approx(r2), kSMaxF);
  if (MASK) s = self ? 0.0f : s;
  r = r2 * s;
  e = ex2_approx(r * c.nkl2e);
}
template <bool MASK>
__device__ __forceinline__ void radial(double r2, bool self, const PairConst<double>& c, double& s,
                                       double& r, double& e) {
  s = fmin(rsqrt(r2), kSMaxD);
  if (MASK) s = self ? 0.0 : s;
  r = r2 * s;
  e = exp(-c.kappa * r);
}

// Forward pair: target (x, n) gathers source (xs, a = ds psi, m = ds phi n).
template <bool MASK, typename T>
__device__ __forceinline__ void pair_forward(T xi, T yi, T zi, T nxi, T nyi, T nzi, T xj, T yj, T zj,
                                             T a, T mx, T my, T mz, bool self, const PairConst<T>& c,
                                             T& accP, T& accQ) {
  T dx = xi - xj, dy = yi - yj, dz = zi - zj;
  T r2 = dx * dx + dy * dy + dz * dz;
  T s, r, e;
  radial<MASK>(r2, self, c, s, r, e);
  T kr = r * c.kappa;
  T ci = nxi * dx + nyi * dy + nzi * dz;
  T cm = mx * dx + my * dy + mz * dz;
  T cim = nxi * mx + nyi * my + nzi * mz;
  T t = e * kr + e;
  T tm1 = t - T(1);
  T wm3 = (t - e) * kr + T(3) * tm1;
  T s2 = s * s;
  // P = s [ (1 - e) a + (eps t - 1) cm s^2 ]
  T p = a - e * a;
  p = ((c.eps * t - T(1)) * cm) * s2 + p;
  accP = p * s + accP;
  // Q = s^3 [ (t/eps - 1) ci a + (t - 1) cim - (w - 3) ci cm s^2 ]
  T q = ((t * c.inveps - T(1)) * ci) * a;
  q = tm1 * cim + q;
  q = q - wm3 * ((ci * cm) * s2);
  accQ = q * (s2 * s) + accQ;
}

// Transposed pair: output element j (x, n) gathers element i (xs, wphi, p = wpsi n_i),
// d = x_i - x_j:
//   Zphi = s^3 [ (eps t - 1) c_j wphi + (t - 1) (n_j.p) - (w - 3) (p.d) c_j s^2 ]
//   Zpsi = s [ (1 - e) wphi + (t/eps - 1) (p.d) s^2 ]
// (K2 and K4 gathered into the phi output, K1 and K3 into the psi output; the
// output element's area ds_j is applied in the reduction.)
template <bool MASK, typename T>
__device__ __forceinline__ void pair_transpose(T xj, T yj, T zj, T nxj, T nyj, T nzj, T xi, T yi, T zi,
                                               T wphi, T px, T py, T pz, bool self,
                                               const PairConst<T>& c, T& accP, T& accQ) {
  T dx = xi - xj, dy = yi - yj, dz = zi - zj;
  T r2 = dx * dx + dy * dy + dz * dz;
  T s, r, e;
  radial<MASK>(r2, self, c, s, r, e);
  T kr = r * c.kappa;
  T cj = nxj * dx + nyj * dy + nzj * dz;
  T cp = px * dx + py * dy + pz * dz;
  T cnp = nxj * px + nyj * py + nzj * pz;
  T t = e * kr + e;
  T tm1 = t - T(1);
  T wm3 = (t - e) * kr + T(3) * tm1;
  T s2 = s * s;
  T q = ((c.eps * t - T(1)) * cj) * wphi;
  q = tm1 * cnp + q;
  q = q - wm3 * ((cp * cj) * s2);
  accP = q * (s2 * s) + accP;
  T p = wphi - e * wphi;
  p = ((t * c.inveps - T(1)) * cp) * s2 + p;
  accQ = p * s + accQ;
}

// ------------------------------------------------------------------ symmetric pairs
// The four kernels depend on the pair through r, e, t, w (symmetric in i and
// j) and through c_i, c_j, c_ij and the sign of d (d_ji = -d_ij).  A kernel
// that visits the unordered pair {i, j} once computes the radial terms once
// and applies them in both directions: target i gathering source j
// (sign +1, d = x_i - x_j) and target j gathering source i (sign -1).
// s = 1/r, s3 = s^3, ome = 1 - e, tm1 = t - 1, wm3s2 = (w - 3) s^2, and
// ka = (eps t - 1) s^2, kb = t/eps - 1 for A u (TRANS = false), or
// ka = eps t - 1, kb = (t/eps - 1) s^2 for A^T w (TRANS = true).
template <typename T>
struct SymTerms {
  T s, s3, ome, tm1, ka, kb, wm3s2;
};

template <bool MASK, bool TRANS, typename T>
__device__ __forceinline__ SymTerms<T> sym_terms(T dx, T dy, T dz, bool self, const PairConst<T>& c) {
  SymTerms<T> R;
  T r, e;
  radial<MASK>(dx * dx + dy * dy + dz * dz, self, c, R.s, r, e);
  const T kr = r * c.kappa;
  const T ekr = e * kr;
  const T t = ekr + e;
  R.tm1 = t - T(1);
  const T s2 = R.s * R.s;
  R.wm3s2 = (ekr * kr + T(3) * R.tm1) * s2;  // w - 3 = 3 (t - 1) + e (kappa r)^2
  R.ome = T(1) - e;
  R.s3 = s2 * R.s;
  const T et1 = c.eps * t - T(1), te1 = t * c.inveps - T(1);
  R.ka = TRANS ? et1 : et1 * s2;
  R.kb = TRANS ? te1 * s2 : te1;
  return R;
}

// Forward direction (R from sym_terms<MASK, false>): target (normal nt) gathers
// source (a = ds psi, m = ds phi n);
// SIGN = +1 when d points from the source to the target, -1 otherwise.
//   P += s [ (1 - e) a + (eps t - 1) (m.d) s^2 ]
//   Q += s^3 [ (t/eps - 1) (nt.d) a + (t - 1) (nt.m) - (w - 3) (nt.d)(m.d) s^2 ]
template <int SIGN, typename T>
__device__ __forceinline__ void sym_forward(const SymTerms<T>& R, T dx, T dy, T dz, T ntx, T nty, T ntz, T a, T mx,
                                            T my, T mz, T& accP, T& accQ) {
  const T ci = ntx * dx + nty * dy + ntz * dz;
  const T cm = mx * dx + my * dy + mz * dz;
  const T cim = ntx * mx + nty * my + ntz * mz;
  T p = R.ome * a;
  p = (T(SIGN) * R.ka) * cm + p;
  accP = p * R.s + accP;
  T q = (T(SIGN) * R.kb * ci) * a;
  q = R.tm1 * cim + q;
  q = q - R.wm3s2 * (ci * cm);
  accQ = q * R.s3 + accQ;
}

// Transposed direction (R from sym_terms<MASK, true>): output element (normal no)
// gathers element (wphi, p = wpsi n);
// SIGN = +1 when d points from the output element to the gathered one.
//   Zphi += s^3 [ (eps t - 1) (no.d) wphi + (t - 1)(no.p) - (w - 3)(p.d)(no.d) s^2 ]
//   Zpsi += s [ (1 - e) wphi + (t/eps - 1)(p.d) s^2 ]
template <int SIGN, typename T>
__device__ __forceinline__ void sym_transpose(const SymTerms<T>& R, T dx, T dy, T dz, T nox, T noy, T noz, T wphi,
                                              T px, T py, T pz, T& accP, T& accQ) {
  const T cj = nox * dx + noy * dy + noz * dz;
  const T cp = px * dx + py * dy + pz * dz;
  const T cnp = nox * px + noy * py + noz * pz;
  T q = (T(SIGN) * R.ka * cj) * wphi;
  q = R.tm1 * cnp + q;
  q = q - R.wm3s2 * (cp * cj);
  accP = q * R.s3 + accP;
  T p = R.ome * wphi;
  p = (T(SIGN) * R.kb) * cp + p;
  accQ = p * R.s + accQ;
}

}  // namespace bipb
