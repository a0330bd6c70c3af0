// Multi-right-hand-side mat-vec on the 5th-generation tensor cores.
//
// Y = A U for a block of up to 64 right-hand sides U (2N x B) on one
// surface.  Per CTA: 128 targets (two MMA tiles of M = 128 rows: tile 0 the
// phi_i rows, tile 1 the psi_i rows of the same targets) against a range of
// source chunks of 16 sources (K = 32 source unknowns phi_j, psi_j
// interleaved).  For every chunk the CUDA cores generate the kernel tile
// once,
//     [ K2 ds_j   K1 ds_j ]        (row phi_i, tile 0)
//     [ K4 ds_j   K3 ds_j ]        (row psi_i, tile 1)     (Sec. 2.2.1, Eqs. 5-6)
// split every FP32 value a into TF32 parts (a_hi: a rounded to 11
// significant bits by Veltkamp's splitting, exact in TF32; a_lo = a - a_hi)
// and write both into tensor memory, where the MMA reads its A operand: the
// thread that owns TMEM lane r owns target r's row in both tiles, so it
// computes a pair's four values once and writes each where it belongs (four
// threads per target, one quarter of the chunk's sources each).  The U tile
// of a chunk (U_hi in rows 0..63, U_lo in rows 64..127, packed per chunk in
// global memory by k_pack_u_tc, K-major core-matrix layout) arrives by a bulk
// copy into shared memory, and one thread issues, per K step of 8 and tile,
// two tcgen05.mma kind::tf32 (M = 128, N = 128, K = 8, A in TMEM, B in shared
// memory): A_hi [U_hi | U_lo] and A_lo [U_hi | U_lo] into one FP32
// accumulator of 128 columns, whose halves are added when it is read back.
// That is A_hi U_hi + A_hi U_lo + A_lo U_hi (+ A_lo U_lo) in two MMAs: an
// M = 128, K = 8 MMA takes as long for N = 128 as for N = 64 (about 96 SM
// cycles measured on GB300), so this takes two thirds of the tensor-core time of three
// N = 64 products.  The MMAs run while the next tile is being generated;
// shared memory carries only the U tiles.
//
// TMEM (512 columns; lane r = target r of the CTA): A buffers 0, 1 at columns
// [0, 128), [128, 256) (tile m at + 64 m: hi part + 0..31, lo part + 32..63);
// the accumulator of tile m at [256 + 128 m, 384 + 128 m).
//
// Accuracy.  The products drop only the TF32 truncation of the low parts,
// about 2^-22 of a product.  The tensor core's FP32 accumulation, however, is
// not to be run over a whole source range: summed over thousands of chunks
// its error grows with the length of the sum and does not average out for
// smooth vectors (measured on the protein-like surface at N = 81920: 1.7e-4
// of the off-diagonal part for phi = 1, against 1.2e-5 for the FP32
// CUDA-core mat-vec).  So every group of eight chunks (K = 256) starts a
// fresh accumulator: the threads read group g back (and add it to FP32
// registers) at the second chunk of group g + 1, whose first MMAs wait for
// that.  The operator is then accurate to FP32 level and the mixed refinement
// reaches 1e-8 in two steps.  The epilogue writes per-split partial sums that
// the FP64 reduction of kernels.cu adds, so the kernel tile costs about the
// same as in the single-RHS kernel while serving 64 right-hand sides.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets an error
// flag that the host turns into BIPB_ERR_CUDA, and the kernel still frees its
// tensor memory.
#include <algorithm>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace bipb {

namespace {

constexpr int kNB = 64;          // right-hand sides per launch (MMA N)
constexpr int kTgt = 128;        // targets per CTA (two M = 128 tiles)
constexpr int kChunk = 16;       // sources per chunk
constexpr int kK = 2 * kChunk;   // MMA K per chunk
constexpr int kBBytes = kNB * kK * 4;       // one TF32 part of the U tile of a chunk: 8 KB
constexpr int kSBytes = kChunk * 32;        // source records of one chunk: 512 B
constexpr int kRing = 8;                    // U and source buffers (chunk it in buffer it % 8)
constexpr int kOffB = 0;                    // kRing U buffers, each [hi | lo]
constexpr int kOffS = kOffB + kRing * 2 * kBBytes;  // kRing source buffers
constexpr int kOffBar = kOffS + kRing * kSBytes;
constexpr int kSmemBytes = kOffBar + (3 * kRing + 8) * 8 + 16;
constexpr int kGroup = 8;                   // chunks accumulated in TMEM before it is read back (16 fails the FP32 bound)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColA = 0;               // A buffer s at kColA + 128 s
constexpr uint32_t kColD = 256;             // accumulator of tile m at kColD + 128 m
constexpr long kSpinLimit = 1L << 24;

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// a rounded to 11 significant bits (Veltkamp's splitting with the factor
// 2^13 + 1), exactly representable in TF32; a - split_hi(a) is exact in FP32.
// The intrinsics keep the compiler from contracting the three operations.
__device__ __forceinline__ float split_hi(float a) {
  const float c = __fmul_rn(a, 8193.0f);
  return __fsub_rn(c, __fsub_rn(c, a));
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

// U (FP64, system b at b * 2n: [phi; psi]) -> per chunk, the TF32 tiles U_hi
// and U_lo (one after the other) in the K-major core-matrix layout (row =
// right-hand side, K = 2 j' + c).
__global__ void k_pack_u_tc(int n, int n_rhs, int n_chunks, const double* __restrict__ u, float* __restrict__ upk) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one per (chunk, b, k)
  if (e >= (int64_t)n_chunks * kNB * kK) return;
  const int ch = (int)(e / (kNB * kK));
  const int rem = (int)(e % (kNB * kK));
  const int b = rem / kK, k = rem % kK;
  const int j = ch * kChunk + (k >> 1), c = k & 1;
  float hi = 0.f, lo = 0.f;
  if (b < n_rhs && j < n) {
    const double v = u[(int64_t)b * 2 * n + (int64_t)c * n + j];
    hi = to_tf32((float)v);
    lo = to_tf32((float)(v - (double)hi));
  }
  float* tile = upk + (int64_t)ch * (2 * kNB * kK);
  tile[tc::kmajor_offset(b, k, kK) / 4] = hi;
  tile[kNB * kK + tc::kmajor_offset(b, k, kK) / 4] = lo;
}

// The four kernel values of pair (target i, source j) times ds_j (times 4 pi),
// in FP32: returns (K2, K1) in v[0], v[1] and (K4, K3) in v[2], v[3].
__device__ __forceinline__ void kernel_block(float xi, float yi, float zi, float nxi, float nyi, float nzi, float4 g,
                                             float4 nv, bool zero, const PairConst<float>& c, float* v) {
  const float dx = xi - g.x, dy = yi - g.y, dz = zi - g.z;
  const float r2 = dx * dx + dy * dy + dz * dz;
  float s = fminf(rsqrt_approx(r2), kSMaxF);
  s = zero ? 0.f : s;
  const float r = r2 * s;
  const float e = ex2_approx(r * c.nkl2e);
  const float kr = r * c.kappa;
  const float ci = nxi * dx + nyi * dy + nzi * dz;
  const float cj = nv.x * dx + nv.y * dy + nv.z * dz;
  const float cij = nxi * nv.x + nyi * nv.y + nzi * nv.z;
  const float t = e * kr + e;
  const float tm1 = t - 1.f;
  const float wm3 = (t - e) * kr + 3.f * tm1;
  const float sa = s * g.w;
  const float s2 = s * s;
  const float s3a = s2 * sa;
  v[1] = sa - e * sa;                                  // K1 ds = (1 - e) s ds
  v[0] = ((c.eps * t - 1.f) * cj) * s3a;               // K2 ds
  v[3] = ((t * c.inveps - 1.f) * ci) * s3a;            // K3 ds
  v[2] = (tm1 * cij - wm3 * ((ci * cj) * s2)) * s3a;   // K4 ds
}

// items: {t0, c0, c1, split}; tgt32: 2 float4 per element (x, y, z, area), (n, 0).
// Warps 0-15 generate tiles and accumulate; warp 16 (one lane) issues the
// bulk copies and the MMAs, so no generating warp waits for the issue.
constexpr int kGenThreads = 512;
constexpr int kMmaWarp = kGenThreads / 32;     // warp 16: issues the MMAs (one lane)
constexpr int kLoadWarp = kMmaWarp + 1;         // warp 17: issues the bulk copies (one lane)
constexpr int kThreads = kGenThreads + 64;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_mrhs_tc(int n, int n_rhs, int n_splits, const int4* __restrict__ items,
                                                    const float4* __restrict__ tgt32, const float* __restrict__ upk,
                                                    float* __restrict__ part, PairConst<float> c,
                                                    int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* ufull = reinterpret_cast<uint64_t*>(smem + kOffBar);  // kRing: U tile of a chunk landed
  uint64_t* sfull = ufull + kRing;                                 // kRing: source records of a chunk landed
  uint64_t* ready = sfull + kRing;                                // 2: A tile of a chunk in TMEM (16 warp arrivals)
  uint64_t* afree = ready + 2;                                    // 2: MMAs of a chunk finished (per A buffer)
  uint64_t* done = afree + 2;                                     // 1: MMAs of a group finished
  uint64_t* drained = done + 1;                                   // 1: accumulators read back (16 warp arrivals)
  uint64_t* bfree = drained + 1;                                  // kRing: MMAs of the buffer's chunk finished
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bfree + kRing);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 item = items[blockIdx.x];
  const int t0 = item.x, c0 = item.y, c1 = item.z, split = item.w;

  if (tid == 0) {
    for (int q = 0; q < kRing; ++q) {
      tc::mbar_init(&ufull[q], 1);
      tc::mbar_init(&sfull[q], 1);
      tc::mbar_init(&bfree[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&ready[q], kGenThreads / 32);
      tc::mbar_init(&afree[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(drained, kGenThreads / 32);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int n_it = c1 - c0;
  const int n_groups = (n_it + kGroup - 1) / kGroup;
  bool ok = true;
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
        if (x >= kRing) ok = ok && tc::mbar_wait(&bfree[q], ((x - kRing) / kRing) & 1, kSpinLimit);
        if (!ok) break;
        const int ch = c0 + x;
        const int cnt = min(kChunk, n - ch * kChunk);
        arrive_expect_tx(&sfull[q], cnt * 32);
        bulk_load(smem + kOffS + q * kSBytes, tgt32 + 2 * (int64_t)ch * kChunk, cnt * 32, &sfull[q]);
        arrive_expect_tx(&ufull[q], 2 * kBBytes);
        bulk_load(smem + kOffB + q * 2 * kBBytes, upk + (int64_t)ch * (2 * kNB * kK), 2 * kBBytes, &ufull[q]);
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- MMA warp
    if (lane == 0) {
      // N = 128: the U tile's hi rows (0..63) and lo rows (64..127) in one operand
      const uint32_t idesc = tc::idesc_tf32(128, 2 * kNB);
      // MMAs p0 .. p1 - 1 of chunk it (p = 2 ks + m: K step ks, tile m)
      auto issue = [&](int it, int p0, int p1) {
        const int s = it & 1, q = it % kRing;
        const bool first = it % kGroup == 0;
        // descriptor of the chunk's first U core matrices; the others differ only
        // in the start-address field (bits 0-13, in 16-byte units, no carry)
        const uint64_t db = tc::smem_desc(tc::smem_u32(smem + kOffB + q * 2 * kBBytes), 128, (kK / 4) * 128);
#pragma unroll
        for (int p = 0; p < 2 * (kK / 8); ++p) {
          if (p < p0 || p >= p1) continue;
          const int ks = p >> 1, m = p & 1;
          const uint32_t dcol = tmem + kColD + m * 128;
          const uint32_t a_hi = tmem + kColA + s * 128 + m * 64 + 8 * ks, a_lo = a_hi + 32;
          const uint64_t b = db + (uint64_t)((256 * ks) >> 4);
          // columns 0..63: A_hi U_hi + A_lo U_hi; 64..127: A_hi U_lo + A_lo U_lo
          tc::mma_tf32_ts(dcol, a_hi, b, idesc, (ks > 0 || !first) ? 1u : 0u);
          tc::mma_tf32_ts(dcol, a_lo, b, idesc, 1u);
        }
      };
      for (int it = 0; it < n_it && ok; ++it) {
        const int g = it / kGroup;
        const bool first = it % kGroup == 0, last = it % kGroup == kGroup - 1 || it == n_it - 1;
        // accumulators: group g - 1 read back; the tile of chunk it in TMEM; its U tile landed
        if (first && g >= 1) ok = ok && tc::mbar_wait(drained, (g - 1) & 1, kSpinLimit);
        ok = ok && tc::mbar_wait(&ready[it & 1], (it >> 1) & 1, kSpinLimit);
        ok = ok && tc::mbar_wait(&ufull[it % kRing], (it / kRing) & 1, kSpinLimit);
        if (!ok) break;
        tc::fence_after_sync();
        issue(it, 0, 8);
        tc::mma_commit(&afree[it & 1]);
        tc::mma_commit(&bfree[it % kRing]);
        if (last) tc::mma_commit(done);
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- generating warps
    // this thread owns TMEM lane r = 32 wq + lane: target r of the CTA, whose phi
    // row is row r of tile 0 and whose psi row is row r of tile 1.  It computes
    // sources 4 sq .. 4 sq + 3 of every chunk and reads back accumulator columns
    // 32 (sq & 1) .. + 31 of tile sq >> 1.
    const int sq = warp >> 2;
    const int ti = t0 + 32 * wq + lane;
    const bool tvalid = ti < n;
    const float4 gi = tgt32[2 * min(ti, n - 1)], ni = tgt32[2 * min(ti, n - 1) + 1];
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
      ok = ok && tc::mbar_wait(done, d & 1, kSpinLimit);
      if (!ok) return;
      tc::fence_after_sync();
      read_back();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(drained);
    };
    int drained_groups = 0;
    for (int it = 0; it < n_it; ++it) {
      const int s = it & 1, q = it % kRing;
      ok = ok && tc::mbar_wait(&sfull[q], (it / kRing) & 1, kSpinLimit);
      // chunk it - 2's MMAs read A buffer s
      if (it >= 2) ok = ok && tc::mbar_wait(&afree[s], ((it - 2) >> 1) & 1, kSpinLimit);
      // the second chunk of group g + 1 reads back group g (its last MMAs were
      // those of chunk it - 2, just waited for) before its tile is generated: the
      // first chunk of group g + 1 waits for it
      const int d = (it % kGroup == 1 && it > kGroup) ? it / kGroup - 1 : -1;
      if (d >= 0) ok = ok && tc::mbar_wait(done, d & 1, kSpinLimit);
      if (!ok) break;
      if (it >= 2) tc::fence_after_sync();
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
      const float4* S = reinterpret_cast<const float4*>(smem + kOffS + q * kSBytes);
      float ph[8], ps[8];  // the phi-row and psi-row values in K order (k = 2 u + c)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int jj = 4 * sq + u;
        float v[4];
        if (edge) {
          const bool z = !tvalid || j0 + jj >= n || j0 + jj == ti;
          kernel_block(gi.x, gi.y, gi.z, ni.x, ni.y, ni.z, S[2 * jj], S[2 * jj + 1], z, c, v);
          if (z) v[0] = v[1] = v[2] = v[3] = 0.f;
        } else {
          kernel_block(gi.x, gi.y, gi.z, ni.x, ni.y, ni.z, S[2 * jj], S[2 * jj + 1], false, c, v);
        }
        ph[2 * u] = v[0], ph[2 * u + 1] = v[1];  // K2, K1
        ps[2 * u] = v[2], ps[2 * u + 1] = v[3];  // K4, K3
      }
      float hi[8];
      const uint32_t acol = tmem + lane_base + kColA + s * 128 + 8 * sq;
#pragma unroll
      for (int x = 0; x < 8; ++x) hi[x] = split_hi(ph[x]);
      tc::tmem_st8(acol, hi);
#pragma unroll
      for (int x = 0; x < 8; ++x) ph[x] -= hi[x];  // the low parts (exact in FP32)
      tc::tmem_st8(acol + 32, ph);
      float hs[8];
#pragma unroll
      for (int x = 0; x < 8; ++x) hs[x] = split_hi(ps[x]);
      tc::tmem_st8(acol + 64, hs);
#pragma unroll
      for (int x = 0; x < 8; ++x) ps[x] -= hs[x];
      tc::tmem_st8(acol + 96, ps);
      tc::tmem_wait_st();
      tc::fence_before_sync();
      // one arrival per warp: 512 arrivals on one barrier word would serialise
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[s]);
    }
    for (int d = drained_groups; ok && d < n_groups; ++d) drain(d);
  }
  const bool all_ok = __syncthreads_and(ok) != 0;
  if (!all_ok && tid == 0) atomicExch(err, 1);

  // epilogue: this thread holds target 32 wq + lane, component sq >> 1 (tile),
  // right-hand sides 32 (sq & 1) .. + 31
  if (all_ok && n_it > 0 && warp < kMmaWarp) {
    const int sq = warp >> 2;
    const int i = t0 + 32 * wq + lane, comp = sq >> 1;
    if (i < n)
#pragma unroll
      for (int x = 0; x < 32; ++x) {
        const int b = 32 * (sq & 1) + x;
        if (b < n_rhs) part[((int64_t)b * n_splits + split) * 2 * n + (int64_t)comp * n + i] = acc[x];
      }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int matvec_tc_block() { return kNB; }

void matvec_tc(Surface* s, const SysLayout& L, const PairConst<float>& c, const double* u, double* y, double dphi,
               double dpsi, const int* skip, int skip_stride) {
  const int n = L.n[0];
  for (int k = 0; k < L.K; ++k)
    BIPB_REQUIRE(L.geo_off[k] == 0 && L.n[k] == n && L.vec_off[k] == 2 * n * k,
                 "the tensor-core mat-vec needs right-hand sides of one surface");
  BIPB_CUDA(cudaFuncSetAttribute(k_mrhs_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mrhs_tc, kThreads, kSmemBytes) != cudaSuccess || occ < 1) {
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
  s->grow(s->upk, (size_t)n_chunks * 2 * kNB * kK);
  s->grow(s->part32, (size_t)std::min(K, kNB) * S * 2 * n);
  if (s->tc_err.cap == 0) {
    s->grow(s->tc_err, 1);
    BIPB_CUDA(cudaMemsetAsync(s->tc_err.p, 0, sizeof(int), s->stream));
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
    k_pack_u_tc<<<(int)((pk + 255) / 256), 256, 0, s->stream>>>(n, nb, n_chunks, ub, s->upk.p);
    BIPB_LAUNCHED(s);
    {
      TimedLaunch tl(s, kTMvTC);
      k_mrhs_tc<<<plan->n_items, kThreads, kSmemBytes, s->stream>>>(n, nb, S, plan->items.p, s->tgt32.p, s->upk.p,
                                                               s->part32.p, c, s->tc_err.p);
      BIPB_LAUNCHED(s);
    }
    launch_reduce_matvec32(s, Lb, tt->second->tab.p, s->part32.p, ub, yb, dphi, dpsi,
                           skip ? skip + (int64_t)b0 * skip_stride : nullptr, skip_stride);
  }
}

}  // namespace bipb
