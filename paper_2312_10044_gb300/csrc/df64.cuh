// Double-float ("df64") arithmetic on the FP32 pipe, and the mat-vec pair
// in that arithmetic.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The operations are built from error-free
// transformations: Knuth's TwoSum, Dekker's FastTwoSum (|a| >= |b|) and the
// FMA-based TwoProduct (see Dekker 1971; Shewchuk 1997; Hida, Li and Bailey
// 2001 for the double-double analogue).  The __f*_rn intrinsics keep the
// compiler from contracting or reassociating them.
//
// GB300 executes FP64 at 2 lanes per SM per cycle against 128 for FP32, so
// a mat-vec pair in df64 (several hundred FP32 instructions) is several
// times faster than the same pair in native FP64 while keeping a relative
// accuracy near 1e-13; it serves as the high-precision residual of the mixed
// solve.
//
// exp(-kappa r) follows Tang's table-driven method (ACM TOMS 15, 1989) with
// a table of 1024 values: x = k L + f, L = ln2/1024, |f| <= L/2 (Cody-Waite
// reduction with L split in three parts, the first of 7 significant bits so
// that k L1 is exact for |k| < 2^17), exp(x) = 2^(k>>10) 2^((k&1023)/1024)
// exp(f).  The table values 2^(j/1024) are df64 (computed on the host,
// copied into shared memory by every CTA).  With |f| <= 3.4e-4 the
// polynomial is short: exp(f) = 1 + f + (f^2/2 + f^3/6), the bracket in
// FP32 (it is below 5.8e-8, so its FP32 rounding is below 2^-46), and the
// truncation f^4/24 is below 6e-16.
// 1/sqrt(r2) is one Newton step in df64 from the MUFU estimate (error
// squared: about 1e-14).
#pragma once
#include <cuda_runtime.h>

namespace bipb {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) { return df{hi, lo}; }

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df{s, e};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return df{p, e};
}
// x + y: exact TwoSum of the leading parts, the trailing parts added in FP32.
// Absolute error about 2^-47 max(|x|, |y|).
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, s.lo);
}
// x + y when the exponent of x.hi is at least that of y.hi (FastTwoSum of
// the leading parts is then exact), e.g. 1 - e for 0 < e <= 1.
__device__ __forceinline__ df df_add_ordered(df x, df y) {
  df s = fast_two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
// 1 - e for 0 <= e <= 1 (e = exp(-kappa r)), and t - 1 for 0 <= t <= 1
// (t = e (1 + kappa r)): the exponent of 1 is the larger one.
__device__ __forceinline__ df df_one_minus(df e) { return df_add_ordered(df{1.0f, 0.0f}, df_neg(e)); }
__device__ __forceinline__ df df_minus_one(df t) { return df_add_ordered(df{-1.0f, 0.0f}, t); }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }
// x + f for a float f
__device__ __forceinline__ df df_add_f(df x, float f) {
  df s = two_sum(x.hi, f);
  s.lo = __fadd_rn(s.lo, x.lo);
  return fast_two_sum(s.hi, s.lo);
}
// Products are left unnormalised: the trailing part (the exact error of the
// leading product plus the cross terms) is below a few ulp of the leading
// part, so the next product or sum takes it as it is at no loss of accuracy
// (a chain of d products has a relative error of about d 2^-46), and the
// renormalising FastTwoSum is paid only in sums, where cancellation can
// shrink the leading part.
__device__ __forceinline__ df df_mul(df x, df y) {
  float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df{p, e};
}
__device__ __forceinline__ df df_mul_f(df x, float f) {
  float p = __fmul_rn(x.hi, f);
  float e = __fmaf_rn(x.hi, f, -p);
  e = __fmaf_rn(x.lo, f, e);
  return df{p, e};
}
__device__ __forceinline__ df df_sqr(df x) {
  float p = __fmul_rn(x.hi, x.hi);
  float e = __fmaf_rn(x.hi, x.hi, -p);
  e = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, e);
  return df{p, e};
}
__device__ __forceinline__ df df_scale(df x, float pow2) { return df{__fmul_rn(x.hi, pow2), __fmul_rn(x.lo, pow2)}; }
__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ df df_from_double(double v) {
  float hi = __double2float_rn(v);
  return df{hi, __double2float_rn(v - (double)hi)};
}
// Dot product of two df 3-vectors: the three leading products are exact
// (TwoProduct), their sum is formed by two TwoSums, every trailing part
// (product errors, cross terms, TwoSum errors) is added in FP32, and one
// FastTwoSum renormalises.  Absolute error about 2^-46 of the largest product.
__device__ __forceinline__ df df_dot3(df ax, df ay, df az, df bx, df by, df bz) {
  const float p0 = __fmul_rn(ax.hi, bx.hi), p1 = __fmul_rn(ay.hi, by.hi), p2 = __fmul_rn(az.hi, bz.hi);
  const float e0 = __fmaf_rn(ax.lo, bx.hi, __fmaf_rn(ax.hi, bx.lo, __fmaf_rn(ax.hi, bx.hi, -p0)));
  const float e1 = __fmaf_rn(ay.lo, by.hi, __fmaf_rn(ay.hi, by.lo, __fmaf_rn(ay.hi, by.hi, -p1)));
  const float e2 = __fmaf_rn(az.lo, bz.hi, __fmaf_rn(az.hi, bz.lo, __fmaf_rn(az.hi, bz.hi, -p2)));
  const df s = two_sum(p0, p1);
  const df t = two_sum(s.hi, p2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, s.lo)), t.lo);
  return fast_two_sum(t.hi, lo);
}
// x^2 + y^2 + z^2 for df components, in the same way as df_dot3.
__device__ __forceinline__ df df_sumsq3(df x, df y, df z) {
  const float p0 = __fmul_rn(x.hi, x.hi), p1 = __fmul_rn(y.hi, y.hi), p2 = __fmul_rn(z.hi, z.hi);
  const float e0 = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, __fmaf_rn(x.hi, x.hi, -p0));
  const float e1 = __fmaf_rn(__fadd_rn(y.hi, y.hi), y.lo, __fmaf_rn(y.hi, y.hi, -p1));
  const float e2 = __fmaf_rn(__fadd_rn(z.hi, z.hi), z.lo, __fmaf_rn(z.hi, z.hi, -p2));
  const df s = two_sum(p0, p1);
  const df t = two_sum(s.hi, p2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, s.lo)), t.lo);
  return fast_two_sum(t.hi, lo);
}

constexpr int kExpTab = 1024;  // entries of the exp table, 2^(j/1024) for j < 1024 (k >> 10 below)

struct DFConst {
  df eps, inveps, kappa;  // eps_out/eps_in, its inverse, kappa
  float l1, l2, l3;       // ln2/1024 = l1 + l2 + l3, l1 with 7 significant bits
  float inv_l;            // 1024/ln2
  const float4* tab;      // device copy of the exp table, two df64 entries per float4
};

// Every thread of the CTA copies its share of the exp table into sh (16-byte
// aligned, kExpTab entries); the caller's next barrier makes it visible.
__device__ __forceinline__ void df_load_exp_table(df* sh, const DFConst& c) {
  float4* s4 = reinterpret_cast<float4*>(sh);
  for (int i = threadIdx.x; i < kExpTab / 2; i += blockDim.x) s4[i] = c.tab[i];
}

// 1/sqrt(r2) for r2 > 0: MUFU estimate, one Newton step in df64.
__device__ __forceinline__ df df_rsqrt(df r2) {
  float s0;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(s0) : "f"(r2.hi));
  // h = r2 * s0^2 (close to 1); s = s0 + s0 (1 - h) / 2
  df h = df_mul(r2, two_prod(s0, s0));
  float d = __fadd_rn(__fsub_rn(1.0f, h.hi), -h.lo);  // 1 - h, exact leading part
  return fast_two_sum(s0, __fmul_rn(__fmul_rn(s0, d), 0.5f));
}

// exp(x) for x <= 0 (x.hi clamped at -80), tab[j] = 2^(j/1024) as df64.
__device__ __forceinline__ df df_exp_neg(df x, const DFConst& c, const df* tab) {
  const float xh = fmaxf(x.hi, -80.0f);
  // k = rint(x / L): adding 1.5 * 2^23 leaves the integer in the low mantissa bits
  const float km = __fmaf_rn(xh, c.inv_l, 12582912.0f);
  const int k = __float_as_int(km) - 0x4B400000;
  const float kf = __fsub_rn(km, 12582912.0f);
  // f = x - k L, with k * l1 exact
  const float f1 = __fmaf_rn(-kf, c.l1, xh);  // exact: |f1| < 0.32 on the grid of ulp(min(|x|, 64))
  df f = two_sum(f1, x.lo);
  f = df_add(f, df_neg(two_prod(kf, c.l2)));
  f.lo = __fmaf_rn(-kf, c.l3, f.lo);
  // exp(f) = 1 + f + q, q = f^2/2 + f^3/6 (+ f f.lo, the trailing part's share of f^2/2)
  const float fh = f.hi;
  const float q = __fmaf_rn(fh, f.lo, __fmul_rn(__fmul_rn(fh, fh), __fmaf_rn(fh, 1.0f / 6.0f, 0.5f)));
  df ef = fast_two_sum(1.0f, fh);  // |f| < 1
  ef = fast_two_sum(ef.hi, __fadd_rn(ef.lo, __fadd_rn(f.lo, q)));
  const df r = df_mul(ef, tab[k & (kExpTab - 1)]);
  return df_scale(r, __int_as_float((127 + (k >> 10)) << 23));  // 2^floor(k / 1024)
}

// Forward pair (the formula of pair_forward in pair.cuh) in df64.
// MASK/self: see pair.cuh (s = 0 for the self pair).
template <bool MASK>
__device__ __forceinline__ void df_pair_forward(const df* xi, const df* ni, const df* xj, df a, const df* m, bool self,
                                                const DFConst& c, const df* tab, df& accP, df& accQ) {
  const df dx = df_sub(xi[0], xj[0]), dy = df_sub(xi[1], xj[1]), dz = df_sub(xi[2], xj[2]);
  const df r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
  df s = df_rsqrt(r2);
  if (MASK && self) s = df{0.0f, 0.0f};
  const df r = df_mul(r2, s);
  const df kr = df_mul(r, c.kappa);
  const df e = df_exp_neg(df_neg(kr), c, tab);
  const df ci = df_dot3(ni[0], ni[1], ni[2], dx, dy, dz);
  const df cm = df_dot3(m[0], m[1], m[2], dx, dy, dz);
  const df cim = df_dot3(ni[0], ni[1], ni[2], m[0], m[1], m[2]);
  const df t = df_add(df_mul(e, kr), e);                           // e (1 + kr)
  const df tm1 = df_minus_one(t);                               // t - 1
  const df wm3 = df_add(df_mul(df_sub(t, e), kr), df_mul_f(tm1, 3.0f));  // w - 3 = 3 (t - 1) + (t - e) kr
  const df s2 = df_sqr(s);
  // P = s [ (1 - e) a + (eps t - 1) cm s^2 ]
  const df ome = df_one_minus(e);
  df p = df_mul(ome, a);
  p = df_add(p, df_mul(df_mul(df_add_f(df_mul(c.eps, t), -1.0f), cm), s2));
  accP = df_add(accP, df_mul(p, s));
  // Q = s^3 [ (t/eps - 1) ci a + (t - 1) cim - (w - 3) ci cm s^2 ]
  df q = df_mul(df_mul(df_add_f(df_mul(t, c.inveps), -1.0f), ci), a);
  q = df_add(q, df_mul(tm1, cim));
  q = df_sub(q, df_mul(wm3, df_mul(df_mul(ci, cm), s2)));
  accQ = df_add(accQ, df_mul(q, df_mul(s2, s)));
}

// Transposed pair (the formula of pair_transpose in pair.cuh) in df64:
// output element j (x, n) gathers element i (xs, wphi, p = wpsi n_i).
template <bool MASK>
__device__ __forceinline__ void df_pair_transpose(const df* xj, const df* nj, const df* xi, df wphi, const df* pv,
                                                  bool self, const DFConst& c, const df* tab, df& accP, df& accQ) {
  const df dx = df_sub(xi[0], xj[0]), dy = df_sub(xi[1], xj[1]), dz = df_sub(xi[2], xj[2]);
  const df r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
  df s = df_rsqrt(r2);
  if (MASK && self) s = df{0.0f, 0.0f};
  const df r = df_mul(r2, s);
  const df kr = df_mul(r, c.kappa);
  const df e = df_exp_neg(df_neg(kr), c, tab);
  const df cj = df_dot3(nj[0], nj[1], nj[2], dx, dy, dz);
  const df cp = df_dot3(pv[0], pv[1], pv[2], dx, dy, dz);
  const df cnp = df_dot3(nj[0], nj[1], nj[2], pv[0], pv[1], pv[2]);
  const df t = df_add(df_mul(e, kr), e);
  const df tm1 = df_minus_one(t);
  const df wm3 = df_add(df_mul(df_sub(t, e), kr), df_mul_f(tm1, 3.0f));
  const df s2 = df_sqr(s);
  // Zphi = s^3 [ (eps t - 1) c_j wphi + (t - 1)(n_j.p) - (w - 3)(p.d) c_j s^2 ]
  df q = df_mul(df_mul(df_add_f(df_mul(c.eps, t), -1.0f), cj), wphi);
  q = df_add(q, df_mul(tm1, cnp));
  q = df_sub(q, df_mul(wm3, df_mul(df_mul(cp, cj), s2)));
  accP = df_add(accP, df_mul(q, df_mul(s2, s)));
  // Zpsi = s [ (1 - e) wphi + (t/eps - 1)(p.d) s^2 ]
  df p = df_mul(df_one_minus(e), wphi);
  p = df_add(p, df_mul(df_mul(df_add_f(df_mul(t, c.inveps), -1.0f), cp), s2));
  accQ = df_add(accQ, df_mul(p, s));
}

}  // namespace bipb

namespace bipb {

// The four kernel values of pair (target i, source j) times ds_j (times 4 pi)
// in df64: k[0] = K2 ds, k[1] = K1 ds, k[2] = K4 ds, k[3] = K3 ds (the 2 x 2
// block that maps (phi_j, psi_j) to the (phi_i, psi_i) rows).  s = 0 for the
// self pair when MASK and self.  TRANS: the block of A^T instead, output
// element i gathering input element j (the transposed pair of pair.cuh, d =
// x_i - x_j): k[0] = K2_ji, k[1] = K4_ji (the phi row), k[2] = K1_ji, k[3] =
// K3_ji (the psi row), i.e. ((1 - eps t) c_i s^3, K4, (1 - e) s,
// (1 - t/eps) c_j s^3), times `area` (the output's area goes on the sums).
template <bool MASK, bool TRANS = false>
__device__ __forceinline__ void df_kernel_block(const df* xi, const df* ni, const df* xj, const df* nj, df area,
                                                bool self, const DFConst& c, const df* tab, df* k) {
  const df dx = df_sub(xi[0], xj[0]), dy = df_sub(xi[1], xj[1]), dz = df_sub(xi[2], xj[2]);
  const df r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
  df s = df_rsqrt(r2);
  if (MASK && self) s = df{0.0f, 0.0f};
  const df r = df_mul(r2, s);
  const df kr = df_mul(r, c.kappa);
  const df e = df_exp_neg(df_neg(kr), c, tab);
  const df ci = df_dot3(ni[0], ni[1], ni[2], dx, dy, dz);
  const df cj = df_dot3(nj[0], nj[1], nj[2], dx, dy, dz);
  const df cij = df_dot3(ni[0], ni[1], ni[2], nj[0], nj[1], nj[2]);
  const df t = df_add(df_mul(e, kr), e);
  const df tm1 = df_minus_one(t);
  const df wm3 = df_add(df_mul(df_sub(t, e), kr), df_mul_f(tm1, 3.0f));
  const df sa = df_mul(s, area);
  const df s2 = df_sqr(s);
  const df s3a = df_mul(s2, sa);
  const df k1 = df_mul(df_one_minus(e), sa);                                          // K1 ds
  const df k4 = df_mul(df_sub(df_mul(tm1, cij), df_mul(wm3, df_mul(df_mul(ci, cj), s2))), s3a);  // K4 ds
  if (!TRANS) {
    k[1] = k1;
    k[0] = df_mul(df_mul(df_add_f(df_mul(c.eps, t), -1.0f), cj), s3a);                // K2 ds
    k[3] = df_mul(df_mul(df_add_f(df_mul(t, c.inveps), -1.0f), ci), s3a);             // K3 ds
    k[2] = k4;
  } else {
    k[0] = df_neg(df_mul(df_mul(df_add_f(df_mul(c.eps, t), -1.0f), ci), s3a));        // K2_ji
    k[1] = k4;                                                                        // K4_ji
    k[2] = k1;                                                                        // K1_ji
    k[3] = df_neg(df_mul(df_mul(df_add_f(df_mul(t, c.inveps), -1.0f), cj), s3a));     // K3_ji
  }
}

// acc += a * b with an exact leading product and an unnormalised trailing
// part (renormalise with fast_two_sum before use).
__device__ __forceinline__ void df_mac(df& acc, df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  const float plo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  const df s = two_sum(acc.hi, p.hi);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, plo));
}

}  // namespace bipb

namespace bipb {

// x + y for x, y >= 0, left unnormalised: the trailing part stays within a
// few ulp of the leading one (no cancellation), which products and a
// following exponent-ordered sum take as it is.
__device__ __forceinline__ df df_add_pos_lazy(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return df{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}

// The symmetric pair of pair.cuh (sym_pair) in df64.  The four accumulators
// are updated lazily (df_mac): renormalise them before use.  SCALED: the
// records are in kappa-scaled units as in sym_pair (kappa r = r2 s, (w - 3)
// s^2 = 3 (t - 1) s^2 + e; the caller rescales the sums); otherwise
// unscaled, for any kappa >= 0.
template <bool MASK, bool TRANS, bool SCALED>
__device__ __forceinline__ void df_sym_pair(const df* d, const df* nt, df at, df alt, const df* ns, df as, df als,
                                            bool self, const DFConst& c, const df* tab, df& Pt, df& Qt, df& Ps,
                                            df& Qs) {
  const df r2 = df_sumsq3(d[0], d[1], d[2]);
  df s = df_rsqrt(r2);
  if (MASK && self) s = df{0.0f, 0.0f};
  const df kr = SCALED ? df_mul(r2, s) : df_mul(df_mul(r2, s), c.kappa);
  const df e = df_exp_neg(df_neg(kr), c, tab);
  const df ekr = df_mul(e, kr);
  const df t = df_add_pos_lazy(ekr, e);  // <= 1: the sum with -1 below is exponent-ordered
  const df tm1 = df_minus_one(t);
  const df s2 = df_sqr(s);
  const df s3 = df_mul(s2, s);
  const df wm3s2 = SCALED ? df_add(df_mul_f(df_mul(tm1, s2), 3.0f), e)
                          : df_mul(df_add(df_mul(ekr, kr), df_mul_f(tm1, 3.0f)), s2);
  const df ome = df_one_minus(e);
  const df et1 = df_add_f(df_mul(c.eps, t), -1.0f), te1 = df_add_f(df_mul(t, c.inveps), -1.0f);
  const df ci = df_dot3(nt[0], nt[1], nt[2], d[0], d[1], d[2]);
  const df cj = df_dot3(ns[0], ns[1], ns[2], d[0], d[1], d[2]);
  const df cij = df_dot3(nt[0], nt[1], nt[2], ns[0], ns[1], ns[2]);
  const df U = df_sub(df_mul(tm1, cij), df_mul(wm3s2, df_mul(ci, cj)));
  // s and s^3 folded into the four coefficients every update uses
  const df ome_s = df_mul(ome, s), et1_s3 = df_mul(et1, s3), te1_s3 = df_mul(te1, s3), U_s3 = df_mul(U, s3);
  if (!TRANS) {
    df_mac(Pt, ome_s, as);
    df_mac(Pt, df_mul(et1_s3, cj), als);
    df_mac(Qt, df_mul(te1_s3, ci), as);
    df_mac(Qt, U_s3, als);
    df_mac(Ps, ome_s, at);
    df_mac(Ps, df_neg(df_mul(et1_s3, ci)), alt);
    df_mac(Qs, df_neg(df_mul(te1_s3, cj)), at);
    df_mac(Qs, U_s3, alt);
  } else {
    df_mac(Pt, U_s3, als);
    df_mac(Pt, df_neg(df_mul(et1_s3, ci)), as);
    df_mac(Qt, ome_s, as);
    df_mac(Qt, df_neg(df_mul(te1_s3, cj)), als);
    df_mac(Ps, U_s3, alt);
    df_mac(Ps, df_mul(et1_s3, cj), at);
    df_mac(Qs, ome_s, at);
    df_mac(Qs, df_mul(te1_s3, ci), alt);
  }
}

}  // namespace bipb

namespace bipb {

// Source term of one (element, charge) pair in df64: target element (x, n),
// charge (y, q), d = x - y:  S1 += q s,  S2 += -q (n.d) s^3  (times 4 pi eps_in).
__device__ __forceinline__ void df_source_pair(const df* x, const df* nv, const df* y, df q, df& s1, df& s2) {
  const df d0 = df_sub(x[0], y[0]), d1 = df_sub(x[1], y[1]), d2 = df_sub(x[2], y[2]);
  const df s = df_rsqrt(df_sumsq3(d0, d1, d2));
  const df qs = df_mul(q, s);
  s1 = df_add(s1, qs);
  const df cn = df_dot3(nv[0], nv[1], nv[2], d0, d1, d2);
  s2 = df_sub(s2, df_mul(df_mul(qs, df_sqr(s)), cn));
}

// Reaction potential at a point y from one element (forward record: x, a =
// ds psi, m = ds phi n), d = y - x (the K1, K2 terms with n_j only):
//   4 pi phi += s [ (1 - e) a + (eps t - 1) (m.d) s^2 ]
__device__ __forceinline__ void df_reaction_pair(const df* y, const df* x, df a, const df* m, const DFConst& c,
                                                 const df* tab, df& acc) {
  const df d0 = df_sub(y[0], x[0]), d1 = df_sub(y[1], x[1]), d2 = df_sub(y[2], x[2]);
  const df r2 = df_sumsq3(d0, d1, d2);
  const df s = df_rsqrt(r2);
  const df kr = df_mul(df_mul(r2, s), c.kappa);
  const df e = df_exp_neg(df_neg(kr), c, tab);
  const df t = df_add(df_mul(e, kr), e);
  const df cm = df_dot3(m[0], m[1], m[2], d0, d1, d2);
  df p = df_mul(df_one_minus(e), a);
  p = df_add(p, df_mul(df_mul(df_add_f(df_mul(c.eps, t), -1.0f), cm), df_sqr(s)));
  acc = df_add(acc, df_mul(p, s));
}

// Potential at a point y in the solvent from one element (forward record: x,
// a = ds psi, m = ds phi n), d = y - x: the exterior representation (Eq.
// eqbim_2) with dphi2/dnu = psi / eps (flux continuity), times 4 pi:
//   4 pi phi += s [ t (m.d) s^2 - (1/eps) e a ]   (-Gk dphi2/dnu + dGk/dnu_y phi)
__device__ __forceinline__ void df_exterior_pair(const df* y, const df* x, df a, const df* m, const DFConst& c,
                                                 const df* tab, df& acc) {
  const df d0 = df_sub(y[0], x[0]), d1 = df_sub(y[1], x[1]), d2 = df_sub(y[2], x[2]);
  const df r2 = df_sumsq3(d0, d1, d2);
  const df s = df_rsqrt(r2);
  const df kr = df_mul(df_mul(r2, s), c.kappa);
  const df e = df_exp_neg(df_neg(kr), c, tab);
  const df t = df_add(df_mul(e, kr), e);
  const df cm = df_dot3(m[0], m[1], m[2], d0, d1, d2);
  const df p = df_sub(df_mul(df_mul(t, cm), df_sqr(s)), df_mul(df_mul(c.inveps, e), a));
  acc = df_add(acc, df_mul(p, s));
}

}  // namespace bipb

namespace bipb {

// Energy row of one (element, charge) pair in df64: element j (x, n), charge
// (y, q), d = y - x (times 4 pi):  cphi += q (eps t - 1)(n.d) s^3,  cpsi += q (1 - e) s.
__device__ __forceinline__ void df_energy_row_pair(const df* x, const df* nv, const df* y, df q, const DFConst& c,
                                                   const df* tab, df& cphi, df& cpsi) {
  const df d0 = df_sub(y[0], x[0]), d1 = df_sub(y[1], x[1]), d2 = df_sub(y[2], x[2]);
  const df r2 = df_sumsq3(d0, d1, d2);
  const df s = df_rsqrt(r2);
  const df kr = df_mul(df_mul(r2, s), c.kappa);
  const df e = df_exp_neg(df_neg(kr), c, tab);
  const df t = df_add(df_mul(e, kr), e);
  const df cj = df_dot3(nv[0], nv[1], nv[2], d0, d1, d2);
  const df s3 = df_mul(df_sqr(s), s);
  df_mac(cphi, df_mul(df_mul(q, df_add_f(df_mul(c.eps, t), -1.0f)), cj), s3);
  df_mac(cpsi, df_mul(q, df_one_minus(e)), s);
}

// Energy gradient at a charge y from one element in df64.  Element record:
// x, a = ds psi, normal n, alpha = ds phi (m = alpha n), lphi, beta = lpsi
// (p = beta n) from the adjoint lam = [lphi; lpsi]; d = y - x, cn = n.d.
// With inv = 1 / eps_in (times 4 pi):
//   v   += s [ (1 - e) a + (eps t - 1) alpha cn s^2 ] + inv s [ lphi + beta cn s^2 ]
//   g_m += Cn n_m + Cd d_m, where
//   Cn = s^3 [ (eps t - 1) alpha + inv beta ]
//   Cd = s^3 [ (t - 1) a - (eps w - 3) alpha cn s^2 - inv (lphi + 3 beta cn s^2) ]
// (the y-gradients of the energy row and of the adjoint-weighted source).
__device__ __forceinline__ void df_grad_pair(const df* y, const df* x, df a, const df* nv, df al, df lphi, df beta,
                                             const DFConst& c, df inv, const df* tab, df& v, df* g) {
  const df d[3] = {df_sub(y[0], x[0]), df_sub(y[1], x[1]), df_sub(y[2], x[2])};
  const df r2 = df_sumsq3(d[0], d[1], d[2]);
  const df s = df_rsqrt(r2);
  const df kr = df_mul(df_mul(r2, s), c.kappa);
  const df e = df_exp_neg(df_neg(kr), c, tab);
  const df ekr = df_mul(e, kr);
  const df t = df_add(ekr, e);
  const df w = df_mul(e, df_add_f(df_mul(kr, df_add_f(kr, 3.0f)), 3.0f));  // e (3 + 3 kr + kr^2)
  const df s2 = df_sqr(s);
  const df s3 = df_mul(s2, s);
  const df cn = df_dot3(nv[0], nv[1], nv[2], d[0], d[1], d[2]);
  const df et1 = df_add_f(df_mul(c.eps, t), -1.0f);
  const df acn_s2 = df_mul(df_mul(al, cn), s2);
  const df bcn_s2 = df_mul(df_mul(beta, cn), s2);
  // potential at y and the adjoint-weighted source
  df_mac(v, df_add(df_mul(df_one_minus(e), a), df_mul(et1, acn_s2)), s);
  df_mac(v, df_mul(inv, df_add(lphi, bcn_s2)), s);
  const df Cn = df_mul(df_add(df_mul(et1, al), df_mul(inv, beta)), s3);
  const df Cd = df_mul(df_sub(df_sub(df_mul(df_minus_one(t), a),
                                     df_mul(df_add_f(df_mul(c.eps, w), -3.0f), acn_s2)),
                              df_mul(inv, df_add(lphi, df_mul_f(bcn_s2, 3.0f)))),
                       s3);
  for (int m = 0; m < 3; ++m) {
    df_mac(g[m], Cn, nv[m]);
    df_mac(g[m], Cd, d[m]);
  }
}

}  // namespace bipb
