// Multi-right-hand-side mat-vec on the 5th-generation tensor cores.
//
// Y = A U for a block of up to 64 right-hand sides U (2N x B) on one
// surface.  Per CTA: 128 targets (two MMA tiles of M = 128 rows: tile 0 the
// phi_i rows, tile 1 the psi_i rows of the same targets) against a range of
// source chunks of 32 sources (K = 64 source unknowns phi_j, psi_j
// interleaved).  For every chunk the CUDA cores generate the kernel tile
// once,
//     [ K2 ds_j   K1 ds_j ]        (row phi_i, tile 0)
//     [ K4 ds_j   K3 ds_j ]        (row psi_i, tile 1)     (Sec. 2.2.1, Eqs. 5-6)
// in FP32 (each column scaled by a power of two through scaled source
// records, below; two sources per packed-FP32 instruction, f32x2.cuh, from
// source records interleaved by pairs), split each value a into two FP16 parts (a_hi = a rounded to FP16, a_lo = a - a_hi rounded to FP16:
// 22 significant bits together) and write both into tensor memory, where the
// MMA reads its A operand: the thread that owns TMEM lane r owns target r's
// row in both tiles, so it computes a pair's four values once and writes each
// where it belongs (four threads per target, one quarter of the chunk's
// sources each).  The U tile of a chunk (U_hi in rows 0..63, U_lo in rows
// 64..127, each row scaled by a power of two; packed per chunk in global
// memory by k_pack_u_tc, K-major core-matrix layout) arrives by a bulk copy
// into shared memory, and one thread issues, per K step of 16 and tile, two
// tcgen05.mma kind::f16 (M = 128, N = 128, K = 16, A in TMEM, B in shared
// memory, FP32 accumulator): A_hi [U_hi | U_lo] and A_lo [U_hi | U_lo] into
// one accumulator of 128 columns, whose halves are added when it is read back.
// That is A_hi U_hi + A_hi U_lo + A_lo U_hi (+ A_lo U_lo) in two MMAs.  On
// GB300 an M = 128, N = 128 MMA takes about 117 SM cycles with K = 16 in FP16
// and 111 with K = 8 in TF32 (measured, one thread issuing back to back), so
// the FP16 split needs half the tensor-core time of a TF32 split of the same
// accuracy.  The MMAs run while the next tile is being generated (two A
// buffers); shared memory carries only the U tiles.
//
// Scaling.  FP16 holds 2^-14 .. 65504 at full precision, so both operands are
// brought to a known range by exact powers of two.  Column (j, c) of A (the
// source unknown phi_j or psi_j) is multiplied by 2^e(j, c), chosen once per
// surface and medium (k_tc_colexp, over all targets) so that its largest
// value lies in [2^14, 2^15); the factors are folded into a scaled copy of
// the source records (area times 2^e(j, 1), normal times 2^(e(j, 0) -
// e(j, 1)): the K2 and K4 values are linear in n_j, the K1 and K3 values do
// not depend on it), so generating a scaled value costs nothing extra.  Row
// (j, c) of U is multiplied by 2^(f(b) - e(j, c)), f(b) chosen per call so
// that the largest scaled value of right-hand side b lies in [2^14, 2^15).
// The epilogue multiplies each sum by 2^-f(b).  A value far below its
// column's (or right-hand side's) largest loses relative precision in its
// low part (FP16 subnormals), but its absolute error stays below 2^-40 of
// that largest value.
//
// TMEM (512 columns; lane r = target r of the CTA): A buffers 0, 1 at columns
// 128 s (tile m at + 64 m: hi part + 0..31, lo part + 32..63, two FP16 values
// per column); the accumulator of tile m at [256 + 128 m, 384 + 128 m).
//
// Accuracy.  The tensor core's FP32 accumulation is not to be run over a
// whole source range: summed over thousands of chunks its error grows with
// the length of the sum and does not average out for smooth vectors
// (measured on the protein-like surface at N = 81920: 1.7e-4 of the
// off-diagonal part for phi = 1, against 1.2e-5 for the FP32 CUDA-core
// mat-vec).  So every group of 128 sources (four chunks, K = 256) starts a
// fresh accumulator: the threads read group g back (and add it to FP32 registers)
// at the second chunk of group g + 1, whose first MMAs wait for that.  The
// operator is then accurate to FP32 level and the mixed refinement reaches
// 1e-8 in two steps.  The epilogue writes per-split partial sums that the
// FP64 reduction of kernels.cu adds, so the kernel tile costs about the same
// as in the single-RHS kernel while serving 64 right-hand sides.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets an error
// flag that the host turns into BIPB_ERR_CUDA, and the kernel still frees its
// tensor memory.
#include <cuda_fp16.h>

#include <algorithm>

#include "f32x2.cuh"
#include "internal.cuh"
#include "tcgen05.cuh"

namespace bipb {

namespace {

constexpr int kNB = 64;                     // right-hand sides per launch (MMA N = 2 kNB: hi and lo parts)
constexpr int kTgt = 128;                   // targets per CTA (two M = 128 tiles)
constexpr int kChunk = 32;                  // sources per chunk
constexpr int kK = 2 * kChunk;              // MMA K per chunk (four K steps of 16)
constexpr int kPerThread = kChunk / 4;      // sources of a chunk per generating thread
constexpr int kPartBytes = kNB * kK * 2;    // one FP16 part of the U tile of a chunk: 8 KB
constexpr int kUBytes = 2 * kPartBytes;     // [U_hi | U_lo] of a chunk: 128 rows of 128 bytes
constexpr int kSBytes = kChunk * 32;        // source records of one chunk: 1 KB
constexpr int kRing = 8;                    // U and source buffers (chunk it in buffer it % 8)
constexpr int kACols = 4 * kChunk;          // TMEM columns of one A buffer: 2 tiles x (hi, lo) x K / 2
constexpr int kABuf = 256 / kACols;         // A buffers in TMEM (chunk it in buffer it % kABuf)
constexpr int kOffB = 0;                    // kRing U buffers
constexpr int kOffS = kOffB + kRing * kUBytes;      // kRing source buffers
constexpr int kOffCol = kOffS + kRing * kSBytes;    // kNB column unscale factors
constexpr int kOffBar = kOffCol + kNB * 4;
constexpr int kNumBars = 3 * kRing + 2 * kABuf + 2;
constexpr int kSmemBytes = kOffBar + kNumBars * 8 + 16;
constexpr int kGroup = 128 / kChunk;        // chunks accumulated in TMEM before it is read back: 128 sources (256 fail the FP32 bound)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColA = 0;               // A buffer s at kColA + kACols s
constexpr uint32_t kColD = 256;             // accumulator of tile m at kColD + 128 m
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // a wait longer than 2 s is an error
constexpr uint64_t kDrainLimitNs = 100000000ull;  // per wait while draining after a time-out
constexpr int kScaleTop = 14;               // scaled magnitudes lie in [2^14, 2^15)
constexpr int kScaleClamp = 100;            // scale exponents are clamped to [-100, 100]
constexpr double kTcKappaMin = 1e-6;        // the kappa-scaled form from this kappa on (1/A)
static_assert(kOffBar % 8 == 0, "mbarriers need 8-byte alignment");

// floor(log2 |x|) of a normal double (-1023 for zero and subnormals, 1024
// for infinities and NaN)
__device__ __forceinline__ int ilog2_bits(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}
// The exponent e that brings a magnitude of floor(log2) lg into [2^14, 2^15)
// by a factor 2^e, clamped to [-100, 100].
__device__ __forceinline__ int scale_exp_lg(int lg) { return max(-kScaleClamp, min(kScaleClamp, kScaleTop - lg)); }
// 2^k for |k| <= 126, and in FP64 for |k| <= 1022
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(127 + k) << 23); }
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// byte offset of element (row, k) of a chunk's FP16 U tile (K = 32, K-major,
// no swizzle): core matrices of 8 rows x 8 values (16 bytes a row)
__host__ __device__ __forceinline__ uint32_t kmajor16_offset(int row, int k) {
  return (uint32_t)((((row >> 3) * (kK >> 3) + (k >> 3)) * 8 + (row & 7)) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}

// colmax[b] = max over sources j and components c of floor(log2 |u_b(j, c)|)
// - e(j, c), at least -1123 for a nonzero u (colmax preset to a value below
// -2000 by a byte fill of 0x80): grid (x, nb)
__global__ void k_colmax_u(int n, const double* __restrict__ u, const int2* __restrict__ srcexp,
                           int* __restrict__ colmax) {
  const int b = blockIdx.y;
  const int64_t len = 2 * (int64_t)n;
  const double* ub = u + (int64_t)b * len;
  int m = INT_MIN;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = ub[e];
    const int j = (int)(e < n ? e : e - n);
    if (v != 0.0) m = max(m, ilog2_bits(v) - (e < n ? srcexp[j].x : srcexp[j].y));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(colmax + b, m);
}

// the scale exponent f(b) of right-hand side b from colmax[b] (100 for a zero column)
__device__ __forceinline__ int rhs_exp(int cm) { return cm < -2000 ? kScaleClamp : scale_exp_lg(cm); }

// U (FP64, system b at b * 2n: [phi; psi]) -> per chunk, u 2^(f(b) - e(j, c))
// split into FP16 parts U_hi (rows 0..63) and U_lo (rows 64..127) in the
// K-major core-matrix layout (row = right-hand side, K = 2 j' + c).
__global__ void k_pack_u_tc(int n, int n_rhs, int n_chunks, const double* __restrict__ u,
                            const int2* __restrict__ srcexp, const int* __restrict__ colmax,
                            __half* __restrict__ upk) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one per (chunk, b, k)
  if (e >= (int64_t)n_chunks * kNB * kK) return;
  const int ch = (int)(e / (kNB * kK));
  const int rem = (int)(e % (kNB * kK));
  const int b = rem / kK, k = rem % kK;
  const int j = ch * kChunk + (k >> 1), c = k & 1;
  __half hi = __float2half_rn(0.f), lo = hi;
  if (b < n_rhs && j < n) {
    const int2 ej = srcexp[j];
    const double v = u[(int64_t)b * 2 * n + (int64_t)c * n + j] * pow2d(rhs_exp(colmax[b]) - (c ? ej.y : ej.x));
    hi = __float2half_rn((float)v);
    lo = __float2half_rn((float)(v - (double)__half2float(hi)));
  }
  unsigned char* tile = reinterpret_cast<unsigned char*>(upk) + (int64_t)ch * kUBytes;
  *reinterpret_cast<__half*>(tile + kmajor16_offset(b, k)) = hi;
  *reinterpret_cast<__half*>(tile + kmajor16_offset(kNB + b, k)) = lo;
}

// The four kernel values of pair (target i, source j) times ds_j (times 4 pi),
// in FP32: returns (K2, K1) in v[0], v[1] and (K4, K3) in v[2], v[3].
// TRANS: the block of A^T instead, output element i gathering input element
// j (pair_transpose of pair.cuh with d = x_i - x_j): the phi row (K2_ji,
// K4_ji) in v[0], v[1], the psi row (K1_ji, K3_ji) in v[2], v[3], times the
// record's area field (the output's area is applied to the sums), i.e.
// ((1 - eps t) c_i s^3, K4, (1 - e) s, (1 - t/eps) c_j s^3).
// SCALED: positions, area and normal in the kappa-scaled units described at
// k_tc_colexp (kappa r = r2 s and (w - 3) s^2 = 3 (t - 1) s^2 + e; one row
// comes out with an extra power of kappa); c.nkl2e and c.smax are then
// -log2(e) and the 1/r cap in those units.
template <bool SCALED, bool TRANS>
__device__ __forceinline__ void kernel_block(float xi, float yi, float zi, float nxi, float nyi, float nzi, float4 g,
                                             float4 nv, bool zero, const PairConst<float>& c, float* v) {
  const float dx = xi - g.x, dy = yi - g.y, dz = zi - g.z;
  const float r2 = dx * dx + dy * dy + dz * dz;
  float s = fminf(rsqrt_approx(r2), c.smax);
  s = zero ? 0.f : s;
  const float r = r2 * s;
  const float e = ex2_approx(r * c.nkl2e);
  const float kr = SCALED ? r : r * c.kappa;
  const float ci = nxi * dx + nyi * dy + nzi * dz;
  const float cj = nv.x * dx + nv.y * dy + nv.z * dz;
  const float cij = nxi * nv.x + nyi * nv.y + nzi * nv.z;
  const float t = e * kr + e;
  const float tm1 = t - 1.f;
  const float sa = s * g.w;
  const float s2 = s * s;
  const float s3a = s2 * sa;
  // (w - 3) s^2
  const float wm3s2 = SCALED ? (3.f * tm1) * s2 + e : ((t - e) * kr + 3.f * tm1) * s2;
  const float k4 = (tm1 * cij - wm3s2 * (ci * cj)) * s3a;
  if (!TRANS) {
    v[1] = sa - e * sa;                                  // K1 ds = (1 - e) s ds
    v[0] = ((c.eps * t - 1.f) * cj) * s3a;               // K2 ds
    v[3] = ((t * c.inveps - 1.f) * ci) * s3a;            // K3 ds
    v[2] = k4;                                           // K4 ds
  } else {
    v[0] = ((1.f - c.eps * t) * ci) * s3a;               // K2_ji
    v[1] = k4;                                           // K4_ji
    v[2] = sa - e * sa;                                  // K1_ji
    v[3] = ((1.f - t * c.inveps) * cj) * s3a;            // K3_ji
  }
}

// kernel_block for the two sources of a record pair at once, in packed FP32
// (two results per instruction).  Source records are pair-interleaved:
// P0 = (x0, x1, y0, y1), P1 = (z0, z1, w0, w1), P2 = (nx0, nx1, ny0, ny1),
// P3 = (nz0, nz1, -, -); T holds the target's x, y, z, nx, ny, nz as splats.
// v[k] holds value k (K2, K1, K4, K3 times ds; for TRANS the transposed
// block in kernel_block's order) of both sources; z0, z1 mask a source as
// `zero` does in kernel_block.
template <bool EDGE, bool SCALED, bool TRANS>
__device__ __forceinline__ void kernel_block2(const f2* T, const float4& P0, const float4& P1, const float4& P2,
                                              const float4& P3, bool z0, bool z1, const PairConst<float>& c, f2* v) {
  const f2 one = f2_splat(1.f), three = f2_splat(3.f);
  const f2 dx = f2_sub(T[0], f2_make(P0.x, P0.y));
  const f2 dy = f2_sub(T[1], f2_make(P0.z, P0.w));
  const f2 dz = f2_sub(T[2], f2_make(P1.x, P1.y));
  const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
  float ra, rb;
  f2_get(r2, ra, rb);
  float sa0 = fminf(rsqrt_approx(ra), c.smax), sb0 = fminf(rsqrt_approx(rb), c.smax);
  if (EDGE) {
    sa0 = z0 ? 0.f : sa0;
    sb0 = z1 ? 0.f : sb0;
  }
  const f2 s = f2_make(sa0, sb0);
  const f2 r = f2_mul(r2, s);
  float ea, eb;
  f2_get(f2_mul(r, f2_splat(c.nkl2e)), ea, eb);
  const f2 e = f2_make(ex2_approx(ea), ex2_approx(eb));
  const f2 kr = SCALED ? r : f2_mul(r, f2_splat(c.kappa));
  const f2 nx = f2_make(P2.x, P2.y), ny = f2_make(P2.z, P2.w), nz = f2_make(P3.x, P3.y);
  const f2 ci = f2_fma(T[3], dx, f2_fma(T[4], dy, f2_mul(T[5], dz)));
  const f2 cj = f2_fma(nx, dx, f2_fma(ny, dy, f2_mul(nz, dz)));
  const f2 cij = f2_fma(T[3], nx, f2_fma(T[4], ny, f2_mul(T[5], nz)));
  const f2 t = f2_fma(e, kr, e);
  const f2 tm1 = f2_sub(t, one);
  const f2 sa = f2_mul(s, f2_make(P1.z, P1.w));
  const f2 s2 = f2_mul(s, s);
  const f2 s3a = f2_mul(s2, sa);
  f2 k4;
  if (SCALED) {  // (w - 3) s^2 = 3 (t - 1) s^2 + e
    const f2 wm3s2 = f2_fma(f2_mul(three, tm1), s2, e);
    k4 = f2_mul(f2_sub(f2_mul(tm1, cij), f2_mul(wm3s2, f2_mul(ci, cj))), s3a);
  } else {
    const f2 wm3 = f2_fma(f2_sub(t, e), kr, f2_mul(three, tm1));
    k4 = f2_mul(f2_sub(f2_mul(tm1, cij), f2_mul(wm3, f2_mul(f2_mul(ci, cj), s2))), s3a);
  }
  const f2 k1 = f2_mul(f2_sub(one, e), sa);
  if (!TRANS) {
    v[1] = k1;                                                                                   // K1 ds
    v[0] = f2_mul(f2_mul(f2_fma(f2_splat(c.eps), t, f2_splat(-1.f)), cj), s3a);                  // K2 ds
    v[3] = f2_mul(f2_mul(f2_fma(t, f2_splat(c.inveps), f2_splat(-1.f)), ci), s3a);               // K3 ds
    v[2] = k4;                                                                                   // K4 ds
  } else {
    v[0] = f2_mul(f2_mul(f2_fma(f2_splat(-c.eps), t, one), ci), s3a);                            // K2_ji
    v[1] = k4;                                                                                   // K4_ji
    v[2] = k1;                                                                                   // K1_ji
    v[3] = f2_mul(f2_mul(f2_fma(t, f2_splat(-c.inveps), one), cj), s3a);                         // K3_ji
  }
}

// Column scale exponents: for source j, e(j, 0) and e(j, 1) from the
// largest magnitude in its phi and psi column (K2 ds_j, K4 ds_j and K1 ds_j,
// K3 ds_j; for A^T the columns of the transposed blocks) over all targets
// i != j (the same FP32 values the tensor-core kernel generates); 0 for a
// column of zeros (no dielectric contrast and kappa = 0), and the two kept
// within 2^40 of each other by lowering the larger, so that the scaled
// normal and the products formed from it stay far from the FP32 range.  Then
// the scaled source records, pair-interleaved for kernel_block2.  One thread
// per source.
//
// A column whose values are linear in the source normal takes its scale
// through the normal, the other through the area field: for A u the phi
// column (K2, K4) is linear in n_j, so the area carries 2^e(j, 1) and the
// normal 2^(e(j, 0) - e(j, 1)); for A^T the psi column (K4, K3) is, and the
// area field (1 instead of ds_j, whose place the output's area takes)
// carries 2^e(j, 0), the normal 2^(e(j, 1) - e(j, 0)).
//
// SCALED (kappa >= kTcKappaMin): positions are multiplied by kappa, and so
// are the source normal and the area field (by kappa^2 for A^T).  With d, r
// and s in Debye lengths the phi row comes out exact and the psi row
// divided (A u) or multiplied (A^T) by kappa, a row factor undone in the
// epilogue, while kappa r = r2 s and (w - 3) s^2 = 3 (t - 1) s^2 + e save
// three FP32 operations per pair.
template <bool SCALED, bool TRANS>
__global__ void __launch_bounds__(128) k_tc_colexp(int n, const float4* __restrict__ tgt32, PairConst<float> c,
                                                   int2* __restrict__ srcexp, float4* __restrict__ src) {
  __shared__ float4 sh[2 * 128];
  const float ks = SCALED ? c.kappa : 1.f;
  const int j = blockIdx.x * 128 + threadIdx.x;
  const int jj = min(j, n - 1);
  float4 gj = tgt32[2 * jj], nj = tgt32[2 * jj + 1];
  gj = make_float4(ks * gj.x, ks * gj.y, ks * gj.z, TRANS ? ks * ks : ks * gj.w);
  nj = make_float4(ks * nj.x, ks * nj.y, ks * nj.z, 0.f);
  float m0 = 0.f, m1 = 0.f;
  for (int i0 = 0; i0 < n; i0 += 128) {
    __syncthreads();
    const int il = min(i0 + (int)threadIdx.x, n - 1);
    sh[2 * threadIdx.x] = tgt32[2 * il];
    sh[2 * threadIdx.x + 1] = tgt32[2 * il + 1];
    __syncthreads();
    const int cnt = min(128, n - i0);
    for (int ii = 0; ii < cnt; ++ii) {
      const float4 g = sh[2 * ii], nv = sh[2 * ii + 1];
      float v[4];
      kernel_block<SCALED, TRANS>(ks * g.x, ks * g.y, ks * g.z, nv.x, nv.y, nv.z, gj, nj, i0 + ii == jj, c, v);
      m0 = fmaxf(m0, fmaxf(fabsf(v[0]), fabsf(v[2])));
      m1 = fmaxf(m1, fmaxf(fabsf(v[1]), fabsf(v[3])));
    }
  }
  if (j >= n) return;
  // floor(log2 m) of a positive normal float
  auto lg = [](float m) { return (int)((__float_as_uint(m) >> 23) & 0xffu) - 127; };
  int e0 = m0 > 0.f ? scale_exp_lg(lg(m0)) : 0, e1 = m1 > 0.f ? scale_exp_lg(lg(m1)) : 0;
  if (e0 - e1 > 40) e0 = e1 + 40;
  if (e1 - e0 > 40) e1 = e0 + 40;
  srcexp[j] = make_int2(e0, e1);
  const float fa = pow2f(TRANS ? e0 : e1), fn = pow2f(TRANS ? e1 - e0 : e0 - e1);
  // pair-interleaved records (kernel_block2): element j in slot j & 1 of pair j >> 1
  float* o = reinterpret_cast<float*>(src) + 16 * (j >> 1) + (j & 1);
  o[0] = gj.x, o[2] = gj.y, o[4] = gj.z, o[6] = gj.w * fa;
  o[8] = nj.x * fn, o[10] = nj.y * fn, o[12] = nj.z * fn, o[14] = 0.f;
}

// two FP32 values (the lower k first) as FP16 parts: hi = round(a), lo =
// round(a - hi).  a - hi comes from one mixed-precision addition of -hi
// (FP16) and a (FP32), exact: |a - hi| is at most half an FP16 unit of hi.
__device__ __forceinline__ void split_f16x2(float a0, float a1, uint32_t& hi, uint32_t& lo) {
  asm("{\n\t.reg .b32 hh;\n\t.reg .f16 h0, h1;\n\t.reg .f32 d0, d1;\n\t"
      "cvt.rn.f16x2.f32 hh, %3, %2;\n\t"
      "mov.b32 {h0, h1}, hh;\n\t"
      "neg.f16 h0, h0;\n\t"
      "neg.f16 h1, h1;\n\t"
      "add.rn.f32.f16 d0, h0, %2;\n\t"
      "add.rn.f32.f16 d1, h1, %3;\n\t"
      "cvt.rn.f16x2.f32 %1, d1, d0;\n\t"
      "mov.b32 %0, hh;\n\t}"
      : "=r"(hi), "=r"(lo)
      : "f"(a0), "f"(a1));
}

// This thread's kPerThread sources of a chunk (pair records Sp, first index
// jq) against target ti (splats T): the scaled pair values, two sources per
// packed evaluation, split into FP16 parts and written into the thread's TMEM
// lane from column acol on (tile 0 hi / lo at + 0 / + kChunk, tile 1 at
// + 2 kChunk / + 3 kChunk).  EDGE masks pairs with no target, a source past
// the end or the self pair.
template <bool EDGE, bool SCALED, bool TRANS>
__device__ __forceinline__ void gen_chunk(const f2* T, const float4* Sp, int jq, int ti, int n, bool tvalid,
                                          const PairConst<float>& c, uint32_t acol) {
#pragma unroll
  for (int hh = 0; hh < kPerThread / 4; ++hh) {
    uint32_t h0[4], l0[4], h1[4], l1[4];  // per source: the phi-row pair (K2, K1) and psi-row pair (K4, K3)
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) {
      const int p = 2 * hh + pp;
      const int ja = jq + 2 * p, jb = ja + 1;
      const bool za = EDGE && (!tvalid || ja >= n || ja == ti), zb = EDGE && (!tvalid || jb >= n || jb == ti);
      f2 v[4];
      kernel_block2<EDGE, SCALED, TRANS>(T, Sp[4 * p], Sp[4 * p + 1], Sp[4 * p + 2], Sp[4 * p + 3], za, zb, c, v);
      float a[4], b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        f2_get(v[k], a[k], b[k]);
        if (EDGE) {
          a[k] = za ? 0.f : a[k];
          b[k] = zb ? 0.f : b[k];
        }
      }
      split_f16x2(a[0], a[1], h0[2 * pp], l0[2 * pp]);
      split_f16x2(a[2], a[3], h1[2 * pp], l1[2 * pp]);
      split_f16x2(b[0], b[1], h0[2 * pp + 1], l0[2 * pp + 1]);
      split_f16x2(b[2], b[3], h1[2 * pp + 1], l1[2 * pp + 1]);
    }
    tc::tmem_st4(acol + 4 * hh, h0);
    tc::tmem_st4(acol + 4 * hh + kChunk, l0);
    tc::tmem_st4(acol + 4 * hh + 2 * kChunk, h1);
    tc::tmem_st4(acol + 4 * hh + 3 * kChunk, l1);
  }
}

// items: {t0, c0, c1, split}; tgt32: 2 float4 per element (x, y, z, area), (n, 0).
// Warp specialisation: warps 0..15 generate the kernel tiles (and read the
// accumulators back), warp 16 issues the MMAs, warp 17 the bulk copies, so no
// generating warp waits for the issue.
constexpr int kGenThreads = 512;
constexpr int kMmaWarp = kGenThreads / 32;     // warp 16: issues the MMAs (one lane)
constexpr int kLoadWarp = kMmaWarp + 1;         // warp 17: issues the bulk copies (one lane)
constexpr int kThreads = kGenThreads + 64;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

template <bool SCALED, bool TRANS>
__global__ void __launch_bounds__(kThreads, 1) k_mrhs_tc(int n, int n_rhs, int n_splits, const int4* __restrict__ items,
                                                    const float4* __restrict__ tgt32, const float4* __restrict__ src,
                                                    const int* __restrict__ colmax,
                                                    const __half* __restrict__ upk, float* __restrict__ part,
                                                    PairConst<float> c, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* ufull = reinterpret_cast<uint64_t*>(smem + kOffBar);  // kRing: U tile of a chunk landed
  uint64_t* sfull = ufull + kRing;                                 // kRing: source records of a chunk landed
  uint64_t* bfree = sfull + kRing;                                 // kRing: MMAs of the buffer's chunk finished
  uint64_t* ready = bfree + kRing;                                 // kABuf: A tile of a chunk in TMEM (16 warp arrivals)
  uint64_t* afree = ready + kABuf;                                 // kABuf: MMAs of a chunk finished (per A buffer)
  uint64_t* done = afree + kABuf;                                  // 1: MMAs of a group finished
  uint64_t* drained = done + 1;                                    // 1: accumulators read back (16 warp arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 1);
  float* cinv = reinterpret_cast<float*>(smem + kOffCol);          // 2^-f(b)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 item = items[blockIdx.x];
  const int t0 = item.x, c0 = item.y, c1 = item.z, split = item.w;

  if (tid == 0) {
    for (int q = 0; q < kRing; ++q) {
      tc::mbar_init(&ufull[q], 1);
      tc::mbar_init(&sfull[q], 1);
      tc::mbar_init(&bfree[q], 1);
    }
    for (int q = 0; q < kABuf; ++q) {
      tc::mbar_init(&ready[q], kGenThreads / 32);
      tc::mbar_init(&afree[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(drained, kGenThreads / 32);
    tc::fence_mbar_init();
  }
  if (tid < kNB) cinv[tid] = pow2f(-rhs_exp(colmax[tid]));
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int n_it = c1 - c0;
  const int n_groups = (n_it + kGroup - 1) / kGroup;
  bool ok = true;
  int issued = 0, mma_last = -1;  // chunks whose copies / MMAs this CTA has issued
  // a generating warp: TMEM lane quarter wq (the warp's own)
  const int wq = warp & 3;
  float acc[32];
#pragma unroll
  for (int x = 0; x < 32; ++x) acc[x] = 0.f;

  if (warp == kLoadWarp) {
    // ---------------------------------------------------------- load warp
    // Chunk x goes into buffer x % kRing once the buffer's previous chunk
    // x - kRing is finished (its MMAs done, which comes after its sources were
    // read: its tile was ready before they ran).  The buffer's next phase needs
    // the copy issued after this wait, so the waits go through every buffer's
    // phases in order.
    if (lane == 0) {
      for (int x = 0; x < n_it; ++x) {
        const int q = x % kRing;
        if (x >= kRing) ok = ok && tc::mbar_wait_timed(&bfree[q], ((x - kRing) / kRing) & 1, kWaitLimitNs);
        if (!ok) break;
        const int ch = c0 + x;
        const int cnt = min(kChunk, n - ch * kChunk);
        arrive_expect_tx(&sfull[q], 64 * ((cnt + 1) / 2));
        // pair records: 64 bytes per pair of sources
        bulk_load(smem + kOffS + q * kSBytes, src + 2 * (int64_t)ch * kChunk, 64 * ((cnt + 1) / 2), &sfull[q]);
        arrive_expect_tx(&ufull[q], kUBytes);
        bulk_load(smem + kOffB + q * kUBytes, reinterpret_cast<const unsigned char*>(upk) + (int64_t)ch * kUBytes,
                  kUBytes, &ufull[q]);
        issued = x + 1;
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- MMA warp
    if (lane == 0) {
      // N = 128: the U tile's hi rows (0..63) and lo rows (64..127) in one operand
      const uint32_t idesc = tc::idesc_f16(128, 2 * kNB);
      for (int it = 0; it < n_it && ok; ++it) {
        const int g = it / kGroup, s = it % kABuf, q = it % kRing;
        const bool first = it % kGroup == 0, last = it % kGroup == kGroup - 1 || it == n_it - 1;
        // accumulators: group g - 1 read back; the tile of chunk it in TMEM; its U tile landed
        if (first && g >= 1) ok = ok && tc::mbar_wait_timed(drained, (g - 1) & 1, kWaitLimitNs);
        ok = ok && tc::mbar_wait_timed(&ready[s], (it / kABuf) & 1, kWaitLimitNs);
        ok = ok && tc::mbar_wait_timed(&ufull[q], (it / kRing) & 1, kWaitLimitNs);
        if (!ok) break;
        tc::fence_after_sync();
        // descriptor of the chunk's U tile: K-direction core matrices 128 bytes
        // apart, 8-row groups kK / 8 core matrices apart; K step ks starts 256 ks
        // bytes further (start-address field, 16-byte units, no carry)
        const uint64_t db = tc::smem_desc(tc::smem_u32(smem + kOffB + q * kUBytes), 128, (kK / 8) * 128);
#pragma unroll
        for (int ks = 0; ks < kK / 16; ++ks)
#pragma unroll
          for (int m = 0; m < 2; ++m) {
            const uint32_t dcol = tmem + kColD + m * 128;
            const uint32_t a_hi = tmem + kColA + s * kACols + m * 2 * kChunk + 8 * ks, a_lo = a_hi + kChunk;
            const uint64_t b = db + (uint64_t)((256 * ks) >> 4);
            // columns 0..63: A_hi U_hi + A_lo U_hi; 64..127: A_hi U_lo + A_lo U_lo
            tc::mma_f16_ts(dcol, a_hi, b, idesc, (ks > 0 || !first) ? 1u : 0u);
            tc::mma_f16_ts(dcol, a_lo, b, idesc, 1u);
          }
        tc::mma_commit(&afree[s]);
        tc::mma_commit(&bfree[q]);
        if (last) tc::mma_commit(done);
        mma_last = it;
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- generating warps
    // this thread owns TMEM lane r = 32 wq + lane: target r of the CTA, whose phi
    // row is row r of tile 0 and whose psi row is row r of tile 1.  It computes
    // sources 8 sq .. 8 sq + 7 of every chunk (A columns 8 sq .. 8 sq + 7 of
    // each part) and reads back accumulator columns 32 (sq & 1) .. + 31 of tile
    // sq >> 1.
    const int sq = warp >> 2;
    const int ti = t0 + 32 * wq + lane;
    const bool tvalid = ti < n;
    const float4 gi = tgt32[2 * min(ti, n - 1)], ni = tgt32[2 * min(ti, n - 1) + 1];
    const float ks = SCALED ? c.kappa : 1.f;  // positions in Debye lengths (k_tc_colexp)
    const f2 T[6] = {f2_splat(ks * gi.x), f2_splat(ks * gi.y), f2_splat(ks * gi.z),
                     f2_splat(ni.x),      f2_splat(ni.y),      f2_splat(ni.z)};
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
    const uint32_t dthr = tmem + lane_base + kColD + (sq >> 1) * 128 + 32 * (sq & 1);
    const bool tile_edge = t0 + kTgt > n;
    auto read_back = [&]() {  // acc += the U_hi and U_lo columns of this thread's 32 right-hand sides
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t v[16], w[16];
        tc::tmem_ld16_async(dthr + 16 * h, v);  // both loads in flight, one wait
        tc::tmem_ld16_async(dthr + 64 + 16 * h, w);
        tc::tmem_wait_ld16(v);
        tc::tmem_wait_ld16(w);
#pragma unroll
        for (int x = 0; x < 16; ++x) acc[16 * h + x] += __uint_as_float(v[x]) + __uint_as_float(w[x]);
      }
    };
    // read-back of a group not read back in the loop (after it); the issue
    // thread may be waiting for it to start the next group
    auto drain = [&](int d) {
      ok = ok && tc::mbar_wait_timed(done, d & 1, kWaitLimitNs);
      if (!ok) return;
      tc::fence_after_sync();
      read_back();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(drained);
    };
    int drained_groups = 0;
    for (int it = 0; it < n_it; ++it) {
      const int s = it % kABuf, q = it % kRing;
      ok = ok && tc::mbar_wait_timed(&sfull[q], (it / kRing) & 1, kWaitLimitNs);
      // chunk it - kABuf's MMAs read A buffer s
      if (it >= kABuf) ok = ok && tc::mbar_wait_timed(&afree[s], ((it - kABuf) / kABuf) & 1, kWaitLimitNs);
      // the second chunk of group g + 1 reads back group g before its tile is
      // generated: the first chunk of group g + 1 waits for it
      const int d = (it % kGroup == 1 && it > kGroup) ? it / kGroup - 1 : -1;
      if (d >= 0) ok = ok && tc::mbar_wait_timed(done, d & 1, kWaitLimitNs);
      if (!ok) break;
      if (it >= kABuf) tc::fence_after_sync();
      if (d >= 0) {
        read_back();
        drained_groups = d + 1;
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(drained);
      }
      const int j0 = (c0 + it) * kChunk;
      // chunks at the end of the surface or over the CTA's own targets, and the
      // last target tile, mask pairs (source past the end, self pair, no target)
      const bool edge = tile_edge || (j0 + kChunk > n) || (j0 < t0 + kTgt && j0 + kChunk > t0);
      const float4* Sp = reinterpret_cast<const float4*>(smem + kOffS + q * kSBytes) + 2 * kPerThread * sq;
      const int jq = j0 + kPerThread * sq;
      const uint32_t acol = tmem + lane_base + kColA + s * kACols + kPerThread * sq;
      // one branch per chunk: the masked form only where a chunk needs it
      if (edge)
        gen_chunk<true, SCALED, TRANS>(T, Sp, jq, ti, n, tvalid, c, acol);
      else
        gen_chunk<false, SCALED, TRANS>(T, Sp, jq, ti, n, tvalid, c, acol);
      tc::tmem_wait_st();
      tc::fence_before_sync();
      // one arrival per warp: 512 arrivals on one barrier word would serialise
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[s]);
    }
    for (int d = drained_groups; ok && d < n_groups; ++d) drain(d);
  }
  const bool all_ok = __syncthreads_and(ok) != 0;
  if (!all_ok) {
    if (tid == 0) atomicExch(err, 1);
    // a wait ran out: the copies and MMAs this CTA issued land before its
    // shared and tensor memory are given up (each wait bounded again)
    if (warp == kLoadWarp && lane == 0)
      for (int x = max(0, issued - kRing); x < issued; ++x) {
        tc::mbar_wait_timed(&sfull[x % kRing], (x / kRing) & 1, kDrainLimitNs);
        tc::mbar_wait_timed(&ufull[x % kRing], (x / kRing) & 1, kDrainLimitNs);
      }
    if (warp == kMmaWarp && lane == 0 && mma_last >= 0)
      tc::mbar_wait_timed(&bfree[mma_last % kRing], (mma_last / kRing) & 1, kDrainLimitNs);
  }

  // epilogue: this thread holds target 32 wq + lane, component sq >> 1 (tile),
  // right-hand sides 32 (sq & 1) .. + 31; the sums are unscaled by 2^-f(b),
  // the psi rows of the kappa-scaled form by kappa (A u) or 1/kappa (A^T),
  // and the sums of A^T take the output element's area
  if (all_ok && n_it > 0 && warp < kMmaWarp) {  // the generating warps
    const int sq = warp >> 2;
    const int i = t0 + 32 * wq + lane, comp = sq >> 1;
    float rowf = (SCALED && comp) ? (TRANS ? 1.f / c.kappa : c.kappa) : 1.f;
    if (TRANS) rowf *= tgt32[2 * min(i, n - 1)].w;
    if (i < n)
#pragma unroll
      for (int x = 0; x < 32; ++x) {
        const int b = 32 * (sq & 1) + x;
        if (b < n_rhs)
          part[((int64_t)b * n_splits + split) * 2 * n + (int64_t)comp * n + i] = acc[x] * (cinv[b] * rowf);
      }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int matvec_tc_block() { return kNB; }

void matvec_tc(Surface* s, const SysLayout& L, const PairConst<float>& c0, bool transpose, const double* u, double* y,
               double dphi, double dpsi, const int* skip, int skip_stride) {
  const int n = L.n[0];
  for (int k = 0; k < L.K; ++k)
    BIPB_REQUIRE(L.geo_off[k] == 0 && L.n[k] == n && L.vec_off[k] == 2 * n * k,
                 "the tensor-core mat-vec needs right-hand sides of one surface");
  // the kappa-scaled form where its 1/r^3 stays far from the FP32 range
  const bool scaled = c0.kappa >= kTcKappaMin;
  PairConst<float> c = c0;
  c.nkl2e = scaled ? -1.4426950408889634f : c0.nkl2e;
  c.smax = scaled ? (float)(kSMaxD / (double)c0.kappa) : kSMaxF;
  auto kernel = scaled ? (transpose ? k_mrhs_tc<true, true> : k_mrhs_tc<true, false>)
                      : (transpose ? k_mrhs_tc<false, true> : k_mrhs_tc<false, false>);
  const int dir = transpose ? 1 : 0;
  BIPB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, kSmemBytes) != cudaSuccess || occ < 1) {
    (void)cudaGetLastError();
    occ = 1;
  }
  const int n_chunks = (n + kChunk - 1) / kChunk;
  const int tiles = (n + kTgt - 1) / kTgt;
  // source splits (whole chunks) that fill whole waves of resident CTAs
  const int slots = s->num_sms * occ;
  int best_s = 1;
  double best = 0.0;
  for (int sp = 1; sp <= std::min(8, std::max(1, n_chunks / 8)); ++sp) {
    const long ctas = (long)tiles * sp, waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / ((double)waves * slots);
    if (eff > best * 1.02) best = eff, best_s = sp;
  }
  const int S = best_s;
  // work list, cached per (n, S)
  const uint64_t key = 0x7c0000000000ull ^ ((uint64_t)n << 8) ^ (uint64_t)S;
  auto it = s->plans.find(key);
  ItemPlan* plan;
  if (it == s->plans.end()) {
    auto p = std::make_unique<ItemPlan>();
    std::vector<int4> items;
    for (int t = 0; t < tiles; ++t)
      for (int sp = 0; sp < S; ++sp)
        items.push_back(make_int4(t * kTgt, (int)((int64_t)sp * n_chunks / S), (int)((int64_t)(sp + 1) * n_chunks / S),
                                  sp));
    p->n_items = (int)items.size();
    p->items.ensure(items.size(), s->stream);
    BIPB_CUDA(cudaMemcpyAsync(p->items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice,
                              s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    ++s->alloc_gen;
    plan = p.get();
    s->plans[key] = std::move(p);
  } else {
    plan = it->second.get();
  }
  const int K = L.K;
  s->grow(s->upk, (size_t)n_chunks * kUBytes / sizeof(float));
  s->grow(s->part32, (size_t)std::min(K, kNB) * S * 2 * n);
  s->grow(s->tc_colmax, (size_t)kNB);
  if (s->tc_err.cap == 0) {
    s->grow(s->tc_err, 1);
    BIPB_CUDA(cudaMemsetAsync(s->tc_err.p, 0, sizeof(int), s->stream));
  }
  // column scale exponents and scaled source records: once per surface and
  // medium (buffers that moved are recomputed)
  const uint64_t gen0 = s->alloc_gen;
  s->grow(s->tc_srcexp[dir], (size_t)n);
  s->grow(s->tc_src[dir], (size_t)4 * ((n + 1) / 2));  // 4 float4 per pair of sources
  int2* srcexp = s->tc_srcexp[dir].p;
  float4* src = s->tc_src[dir].p;
  float* key3 = s->tc_src_key[dir];
  if (s->alloc_gen != gen0 || s->tc_src_n[dir] != n || key3[0] != c.eps || key3[1] != c.inveps ||
      key3[2] != c.kappa) {
    const int nbk = (n + 127) / 128;
    if (scaled && transpose)
      k_tc_colexp<true, true><<<nbk, 128, 0, s->stream>>>(n, s->tgt32.p, c, srcexp, src);
    else if (scaled)
      k_tc_colexp<true, false><<<nbk, 128, 0, s->stream>>>(n, s->tgt32.p, c, srcexp, src);
    else if (transpose)
      k_tc_colexp<false, true><<<nbk, 128, 0, s->stream>>>(n, s->tgt32.p, c, srcexp, src);
    else
      k_tc_colexp<false, false><<<nbk, 128, 0, s->stream>>>(n, s->tgt32.p, c, srcexp, src);
    BIPB_LAUNCHED(s);
    s->tc_src_n[dir] = n;
    key3[0] = c.eps, key3[1] = c.inveps, key3[2] = c.kappa;
  }
  // per block of up to 64 right-hand sides: pack, tensor-core pass, FP64 reduction
  for (int b0 = 0; b0 < K; b0 += kNB) {
    const int nb = std::min(kNB, K - b0);
    std::vector<int> go(nb, 0), nn(nb, n), co(nb, 0), nc(nb, 0);
    SysLayout Lb = make_layout(go, nn, co, nc);
    std::vector<int4> tab(nb);
    for (int b = 0; b < nb; ++b) tab[b] = make_int4(n, S, b * S * 2 * n, 0);
    const uint64_t tkey = 0x7d0000000000ull ^ ((uint64_t)n << 16) ^ ((uint64_t)S << 8) ^ (uint64_t)nb;
    auto tt = s->plans.find(tkey);
    if (tt == s->plans.end()) {
      auto p = std::make_unique<ItemPlan>();
      p->tab.ensure(nb, s->stream);
      BIPB_CUDA(cudaMemcpyAsync(p->tab.p, tab.data(), nb * sizeof(int4), cudaMemcpyHostToDevice, s->stream));
      BIPB_CUDA(cudaStreamSynchronize(s->stream));
      ++s->alloc_gen;
      tt = s->plans.emplace(tkey, std::move(p)).first;
    }
    const double* ub = u + (int64_t)b0 * 2 * n;
    double* yb = y + (int64_t)b0 * 2 * n;
    const int64_t pk = (int64_t)n_chunks * kNB * kK;
    __half* upk = reinterpret_cast<__half*>(s->upk.p);
    BIPB_CUDA(cudaMemsetAsync(s->tc_colmax.p, 0x80, kNB * sizeof(int), s->stream));
    k_colmax_u<<<dim3((unsigned)std::min<int64_t>(64, (2 * (int64_t)n + 255) / 256), nb), 256, 0, s->stream>>>(
        n, ub, srcexp, s->tc_colmax.p);
    BIPB_LAUNCHED(s);
    k_pack_u_tc<<<(int)((pk + 255) / 256), 256, 0, s->stream>>>(n, nb, n_chunks, ub, srcexp,
                                                                  s->tc_colmax.p, upk);
    BIPB_LAUNCHED(s);
    {
      TimedLaunch tl(s, kTMvTC);
      kernel<<<plan->n_items, kThreads, kSmemBytes, s->stream>>>(n, nb, S, plan->items.p, s->tgt32.p,
                                                               src, s->tc_colmax.p, upk, s->part32.p, c,
                                                               s->tc_err.p);
      BIPB_LAUNCHED(s);
    }
    launch_reduce_matvec32(s, Lb, tt->second->tab.p, s->part32.p, ub, yb, dphi, dpsi,
                           skip ? skip + (int64_t)b0 * skip_stride : nullptr, skip_stride);
  }
}

}  // namespace bipb
