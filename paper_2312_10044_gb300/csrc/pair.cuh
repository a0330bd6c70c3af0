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

constexpr float kSMaxF = 1.0e6f;   // 1/r is capped at its value at 1e-6 A (an overflow guard, not a model)
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
  T smax;    // clamp of 1/r in the units of the symmetric pair (1e6 / kappa when scaled by kappa)
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

// Precision-generic pieces of the symmetric pair: 1/sqrt (MUFU estimate in
// FP32), min, and exp(-x) for x >= 0 (MUFU ex2 in FP32).
__device__ __forceinline__ float rsqrt_of(float x) { return rsqrt_approx(x); }
__device__ __forceinline__ double rsqrt_of(double x) { return rsqrt(x); }
__device__ __forceinline__ float min_of(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double min_of(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float exp_neg_of(float x) { return ex2_approx(x * -1.4426950408889634f); }
__device__ __forceinline__ double exp_neg_of(double x) { return exp(-x); }

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
// j) and through c_i = n_i.d, c_j = n_j.d, c_ij = n_i.n_j (d = x_i - x_j, so
// d_ji = -d).  A kernel that visits the unordered pair {i, j} once computes
// them once and applies them in both directions.  With each element's record
// holding its normal, write m = alpha n (alpha = ds phi for A u; for A^T w
// the record's second field p = beta n with beta = wpsi): then m_j.d =
// alpha_j c_j, n_i.m_j = alpha_j c_ij, and both directions share
//   U = (t - 1) c_ij - (w - 3) s^2 c_i c_j.
// A u (a = ds psi):
//   P_i += s [ (1 - e) a_j + (eps t - 1) s^2 alpha_j c_j ]
//   Q_i += s^3 [ (t/eps - 1) c_i a_j + alpha_j U ]
//   P_j += s [ (1 - e) a_i - (eps t - 1) s^2 alpha_i c_i ]
//   Q_j += s^3 [ -(t/eps - 1) c_j a_i + alpha_i U ]
// A^T w (a = wphi; the phi output gathers K2, K4, the psi output K1, K3):
//   Zphi_i += s^3 [ -(eps t - 1) c_i a_j + beta_j U ]
//   Zpsi_i += s [ (1 - e) a_j - (t/eps - 1) s^2 beta_j c_j ]
//   Zphi_j += s^3 [ (eps t - 1) c_j a_i + beta_i U ]
//   Zpsi_j += s [ (1 - e) a_i + (t/eps - 1) s^2 beta_i c_i ]
// (t = target i of the thread, s = source j; P/Q the two outputs of each.)
// Two forms, chosen per launch:
// - SCALED (kappa > 0): positions are multiplied by kappa when the records
//   are packed, so d, r and s are in units of the Debye length; then
//   kappa r = r2 s and (w - 3) s^2 = 3 (t - 1) s^2 + e (with r s = 1).  The
//   kernels scale as K1 ~ kappa, K2, K3 ~ kappa^2, K4 ~ kappa^3, a product of
//   a row factor and a column factor: the records' alpha is multiplied by
//   kappa as well, and the caller multiplies the sums (A u: P by kappa, Q by
//   kappa^2; A^T w: P by kappa^2, Q by kappa).
// - LAPLACE (kappa = 0, unscaled): e = t = 1, w = 3, so K1 = K4 = 0 and only
//   the double-layer terms (eps - 1) c_j s^3 and (1/eps - 1) c_i s^3 remain.
template <bool MASK, bool TRANS, bool LAPLACE, typename T>
__device__ __forceinline__ void sym_pair(T dx, T dy, T dz, const T* nt, T at, T alt, const T* ns, T as, T als,
                                         bool self, const PairConst<T>& c, T& Pt, T& Qt, T& Ps, T& Qs) {
  const T r2 = dx * dx + dy * dy + dz * dz;
  T s = min_of(rsqrt_of(r2), c.smax);
  if (MASK) s = self ? T(0) : s;
  const T ci = nt[0] * dx + nt[1] * dy + nt[2] * dz;
  const T cj = ns[0] * dx + ns[1] * dy + ns[2] * dz;
  const T s3 = s * s * s;
  if constexpr (LAPLACE) {
    const T et1_s3 = c.eps * s3 - s3, te1_s3 = c.inveps * s3 - s3;  // (eps - 1) s^3, (1/eps - 1) s^3
    if (!TRANS) {
      Pt = (et1_s3 * cj) * als + Pt;
      Qt = (te1_s3 * ci) * as + Qt;
      Ps = Ps - (et1_s3 * ci) * alt;
      Qs = Qs - (te1_s3 * cj) * at;
    } else {
      Pt = Pt - (et1_s3 * ci) * as;
      Qt = Qt - (te1_s3 * cj) * als;
      Ps = (et1_s3 * cj) * at + Ps;
      Qs = (te1_s3 * ci) * alt + Qs;
    }
  } else {
    const T kr = r2 * s;  // kappa r (0 for a masked pair)
    const T e = exp_neg_of(kr);
    const T t = e * kr + e;
    const T tm1 = t - T(1);
    const T s2 = s * s;
    // (w - 3) s^2 = 3 (t - 1) s^2 + e (a masked pair gets e = 1, but its every coefficient carries s = 0)
    const T wm3s2 = tm1 * (T(3) * s2) + e;
    const T ts3 = t * s3;
    const T cij = nt[0] * ns[0] + nt[1] * ns[1] + nt[2] * ns[2];
    const T U = tm1 * cij - wm3s2 * (ci * cj);
    // s and s^3 folded into the four coefficients every update uses
    const T ome_s = s - e * s, U_s3 = U * s3;
    const T et1_s3 = c.eps * ts3 - s3, te1_s3 = c.inveps * ts3 - s3;  // (eps t - 1) s^3, (t/eps - 1) s^3
    if (!TRANS) {
      Pt = (et1_s3 * cj) * als + (ome_s * as + Pt);
      Qt = U_s3 * als + ((te1_s3 * ci) * as + Qt);
      Ps = ome_s * at - ((et1_s3 * ci) * alt - Ps);
      Qs = U_s3 * alt - ((te1_s3 * cj) * at - Qs);
    } else {
      Pt = U_s3 * als - ((et1_s3 * ci) * as - Pt);
      Qt = ome_s * as - ((te1_s3 * cj) * als - Qt);
      Ps = U_s3 * alt + ((et1_s3 * cj) * at + Ps);
      Qs = ome_s * at + ((te1_s3 * ci) * alt + Qs);
    }
  }
}
}  // namespace bipb
