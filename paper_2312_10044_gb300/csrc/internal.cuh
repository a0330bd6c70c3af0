// Internal declarations of libbipb (not part of the C ABI).
#pragma once
#include <utility>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <array>
#include <cstring>
#include <vector>

#include "bipb.h"
#include "df64.cuh"
#include "pair.cuh"

namespace bipb {

struct Error : std::runtime_error {
  bipb_status st;
  Error(bipb_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

#define BIPB_CUDA(call)                                                                          \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      throw ::bipb::Error(e_ == cudaErrorMemoryAllocation ? BIPB_ERR_OOM : BIPB_ERR_CUDA,        \
                          std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)
// After every kernel launch: check the launch and count it (a launch issued
// while a graph is being recorded counts toward the graph, not the handle).
#define BIPB_LAUNCHED(sf)                     \
  do {                                        \
    BIPB_CUDA(cudaGetLastError());            \
    if ((sf)->recording)                      \
      ++(sf)->recorded_launches;              \
    else                                      \
      ++(sf)->launches;                       \
  } while (0)
// Programmatic dependent launch along the chain of one Krylov step (record
// pack, pair kernel, reduction, Gram-Schmidt passes, normalisation): each of
// these kernels is launched with launch_chained and begins with
// chain_wait(), which returns once the previous kernel in the stream has
// completed and its writes are visible (at once when there is none or it
// was launched without the attribute); only then does it call
// chain_release(), which lets the next kernel of the chain be scheduled.
// The next kernel's launch and block placement thus overlap this kernel's
// run, while at most two grids of the chain are in flight (a grid is
// released only once every block of its predecessor has passed the wait).
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void chain_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
void launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                    Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BIPB_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

#define BIPB_REQUIRE(cond, msg)                                     \
  do {                                                              \
    if (!(cond)) throw ::bipb::Error(BIPB_ERR_INVALID_ARG, (msg));  \
  } while (0)

// Keep freed device memory in the device's stream-ordered pool (up to this
// many bytes) so that new handles and growing buffers reuse it instead of
// going back to the driver.  Set once per device, for this process only.
void keep_pool_memory(int device);

// Owning device buffer that only grows.  Memory comes from the device's
// stream-ordered pool on the stream that uses the buffer (the handle's), and
// goes back to it on the same stream, ordered after every earlier use.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;
  cudaStream_t stream = nullptr;
  // returns true when the buffer moved
  bool ensure(size_t count, cudaStream_t st = nullptr) {
    if (count <= cap) return false;
    // buffers are created before a CUDA graph is recorded, never inside one
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BIPB_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) throw Error(BIPB_ERR_CUDA, "device buffer allocation while recording a graph");
    release();
    stream = st;
    BIPB_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), stream));
    cap = count;
    return true;
  }
  void release() {
    if (p) cudaFreeAsync(p, stream);
    p = nullptr;
    cap = 0;
  }
  ~DevBuf() { release(); }
};

// The centred centroids of one surface, in FP64 and rounded to FP32, with a
// hash set (open addressing, one flat table of element indices) keyed by the
// bit patterns of the FP32 triple.  FP32 duplicates are found on insertion;
// an FP64 comparison is made only on a key hit.
struct CentroidSet {
  std::vector<double> d;      // 3 per element, FP64
  std::vector<float> f;       // 3 per element, the same rounded to FP32
  std::vector<int32_t> slot;  // element index, or -1
  uint64_t mask = 0;
  static uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  }
  static uint32_t bits(float v) {  // -0 and +0 alike
    uint32_t u;
    const float w = v == 0.0f ? 0.0f : v;
    std::memcpy(&u, &w, 4);
    return u;
  }
  static uint64_t hash(const float* p) {
    return mix(((uint64_t)bits(p[0]) << 32 | bits(p[1])) ^ mix(bits(p[2])));
  }
  static bool same(const float* a, const float* b) {
    return bits(a[0]) == bits(b[0]) && bits(a[1]) == bits(b[1]) && bits(a[2]) == bits(b[2]);
  }
  void reserve(size_t n) {
    size_t sz = 16;
    while (sz < 2 * n) sz <<= 1;
    slot.assign(sz, -1);
    mask = sz - 1;
  }
  // element i (whose f is set) into the table; -1, or the element with the same FP32 point
  int32_t insert(int32_t i) {
    const float* p = &f[3 * (size_t)i];
    for (uint64_t h = hash(p) & mask;; h = (h + 1) & mask) {
      const int32_t j = slot[h];
      if (j < 0) {
        slot[h] = i;
        return -1;
      }
      if (same(&f[3 * (size_t)j], p)) return j;
    }
  }
  // the element at FP32 point p, or -1
  int32_t find(const float* p) const {
    if (slot.empty()) return -1;
    for (uint64_t h = hash(p) & mask;; h = (h + 1) & mask) {
      const int32_t j = slot[h];
      if (j < 0) return -1;
      if (same(&f[3 * (size_t)j], p)) return j;
    }
  }
};


// K independent systems handled by one batched pass (several right-hand
// sides of one surface, or several surfaces).  System k has n[k] elements
// starting at geometry element geo_off[k], 2 n[k] unknowns starting at
// vec_off[k] of a batched vector, and nc[k] charges starting at charge
// record chg_off[k].
struct SysLayout {
  int K = 0;
  std::vector<int> geo_off, n, vec_off, chg_off, nc;
  int64_t len = 0;  // sum of 2 n[k]
  int max_n = 0, max_nc = 0;
  uint64_t key = 0;
};
SysLayout make_layout(const std::vector<int>& geo_off, const std::vector<int>& n, const std::vector<int>& chg_off,
                      const std::vector<int>& nc);

// Work list of one pass (see kernels.cu): items of two int4 each and a
// per-system table {n_tgt, splits, partial offset, 0} for the reductions.
struct ItemPlan {
  DevBuf<int4> items, tab;
  int n_items = 0;
  int64_t part_len = 0;  // partial sums the pass writes
};

// FP32 mat-vec kernel variants (threads per CTA, targets per thread,
// sources per shared-memory chunk): every ordered pair: 0 (256,2,128)
// 1 (256,1,128) 2 (128,2,128) 3 (256,4,128) 4 (128,4,64) 5 (512,1,128)
// 6 (256,2,64); every unordered pair once (sym.cu): 7 (256,2,64)
// 8 (128,4,64) 9 (256,4,64, two CTAs per SM).
constexpr int kNumMv32Variants = 10;
constexpr int kFirstSymVariant = 7;

constexpr int kMaxRestart = 200;

// Per-kernel CUDA-event timing of the pair kernels (off by default).
enum TimedKind { kTMv64 = 0, kTMv32, kTMv64T, kTMv32T, kTSource, kTReaction, kTRow, kTGrad, kTMvDF, kTMvDFT, kTMvTC,
                 kTPotential, kTMvTree, kTKinds };

struct EventPair {
  int kind;
  cudaEvent_t a, b;
};

struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<EventPair> pending;   // recorded by direct launches, read once
  std::vector<EventPair>* capture = nullptr;  // while recording a graph: where its pairs go
  double total_ms[kTKinds] = {0};
  long long count[kTKinds] = {0};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    BIPB_CUDA(cudaEventCreate(&e));
    return e;
  }
  // accumulate finished pairs (the stream has been synchronised)
  void add(const EventPair& p) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      total_ms[p.kind] += ms;
      count[p.kind] += 1;
    } else {
      (void)cudaGetLastError();  // do not leave the failure for the next launch check
    }
  }
  void collect() {
    for (auto& p : pending) {
      add(p);
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void reset() {
    for (int k = 0; k < kTKinds; ++k) total_ms[k] = 0, count[k] = 0;
  }
  ~KernelTimer() {
    for (auto e : pool) cudaEventDestroy(e);
    for (auto& p : pending) cudaEventDestroy(p.a), cudaEventDestroy(p.b);
  }
};

struct GmresWork;  // gmres.cu

// Far-field (treecode) FP32 mat-vec of one surface (tree.cu): the tree, the
// interaction lists cut into balanced work items, and the per-pass scratch.
// Built on first use for the handle's parameters and kept until they change.
struct FarField {
  double theta = 0.0;
  int degree = 0, leaf = 0;
  int n = 0;           // elements
  int n_leaves = 0;    // target batches
  int lmax = 0;        // largest leaf
  int nt = 0;          // threads per CTA of the far-field kernel (lmax rounded up to a warp)
  int n_slots = 0;     // clusters that carry proxy sources
  int n_items = 0;     // work items of the far-field kernel
  int n_up = 0;        // pieces of the upward (proxy weight) pass
  int rec_stride = 0;  // records per system: n elements + n_slots (degree+1)^3 proxies
  int64_t pair_evals = 0;  // (target, record) pairs one mat-vec evaluates per system
  DevBuf<int> perm;        // tree position -> element
  DevBuf<int> leaf_of;     // tree position -> leaf
  DevBuf<int4> leaf_tab;   // per leaf {first position, count, first item, items}
  DevBuf<int4> items;      // per item {leaf, first segment, end segment, 0}
  DevBuf<int2> segs;       // per segment {first record, count}
  DevBuf<int4> up_pieces;  // per upward piece {slot, first position, count, 0}
  DevBuf<int2> up_tab;     // per slot {first piece, pieces}
  DevBuf<float> nodes;     // per slot 3 x (degree+1) Chebyshev nodes, centred FP32
  DevBuf<float4> rec;      // records, 2 float4 each, rec_stride per system
  DevBuf<float> part;      // partial sums, 2 lmax per item and system
  DevBuf<double> upart;    // partial proxy weights, 4 (degree+1)^3 per piece and system
};

struct Surface {
  uint64_t magic = 0;
  int device = 0;
  int num_sms = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;  // private, non-blocking; joined to user_stream per call
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;

  int64_t n = 0;  // elements (all surfaces of a batch handle)

  // Geometry of every element, each surface relative to its own mean
  // centroid (part_center), so that the FP32 copies keep the most digits.
  DevBuf<double4_32a> tgt64;  // 2n: (x, y, z, area), (nx, ny, nz, 0)
  DevBuf<float4> tgt32;   // the same in FP32
  DevBuf<float4> exptab;  // 2^(j/1024), j < 1024, as df64 (hi, lo) pairs: the df64 exp table

  // per-pass scratch
  DevBuf<float4> rec32;
  DevBuf<float4> recdf;
  DevBuf<float> upk;   // FP16 right-hand-side tiles of the tensor-core mat-vec (raw storage)
  DevBuf<int> tc_err;  // set by the tensor-core kernel when a bounded wait ran out
  DevBuf<int> tc_colmax;    // tensor-core mat-vec: per right-hand side, max over sources of log2|u| - e
  // tensor-core mat-vec, per direction (0: A u, 1: A^T u): the scale exponents e
  // of each source's phi and psi columns, the source records with the column
  // scales folded in, and the medium (eps, 1/eps, kappa) and size they were
  // computed for
  DevBuf<int2> tc_srcexp[2];
  DevBuf<float4> tc_src[2];
  float tc_src_key[2][3] = {{0.f, 0.f, -1.f}, {0.f, 0.f, -1.f}};
  int tc_src_n[2] = {-1, -1};
  DevBuf<double4_32a> rec64;
  DevBuf<float> part32;
  DevBuf<double> part64;
  DevBuf<int> rhs_idx;  // right-hand-side indices of a compacted multi-RHS pass
  DevBuf<float4> geodf;  // multi-RHS df64 pass: geometry as df64 records (4 float4 each)
  DevBuf<float4> udf;    // multi-RHS df64 pass: right-hand sides as df64 (phi, psi) pairs
  DevBuf<int2> tcx_rowexp[2];  // exact tensor-core df64 pass, per direction (A u, A^T u): row scale exponents (phi, psi row)
  DevBuf<unsigned> tcx_colmax;  // exact tensor-core df64 pass: max |u| per right-hand side (FP32 bits)
  DevBuf<float> tcx_upk;     // exact tensor-core df64 pass: digit tiles of the right-hand sides (raw storage)
  DevBuf<int> tcx_err;       // set by the exact tensor-core kernel when a bounded wait ran out
  float tcx_key[2][4] = {{0.f, 0.f, -1.f, 0.f}, {0.f, 0.f, -1.f, 0.f}};  // the medium (eps, kappa as df64) of tcx_rowexp
  int tcx_n[2] = {-1, -1};
  DevBuf<double4_32a> pts, pts2;  // points of bipb_potential_at: (p, 0); (p, 0), (0, 0)
  DevBuf<double> pot;             // their potentials, n_rhs x n_pts
  DevBuf<double> coul;            // Coulomb block sums
  DevBuf<int4> coul_tab;          // {0, 0, nc, chg_off} per system

  // charges: every system's charge records (y - center, q), back to back
  int64_t nc = 0;  // charges per configuration (single surface)
  int n_rhs = 0;   // configurations (systems)
  int n_pos_sets = 0;
  DevBuf<double4_32a> chg;
  DevBuf<float4> chgdf;  // the charges as df64 records (2 float4 each), packed by the source pass
  // charges passed on the device (bipb_charges_set_dev): the centroid hash
  // table on the device for the on-centroid check, and the check's flag,
  // read by the next call that uses the charges
  DevBuf<int32_t> key_slots;
  DevBuf<int> chg_err;
  bool chg_check_pending = false;
  SysLayout lay;   // the systems bipb_solve works on

  // surfaces of the handle (one for bipb_surface_create, several for a
  // batch handle, one system each): element offsets, sizes, centres
  std::vector<int> part_off, part_n;
  std::vector<double> part_center;  // 3 per surface
  std::vector<CentroidSet> part_keys;  // the centred centroids of every surface
  std::vector<double> raw_centroids;   // single-surface handles: the centroids as given (tree of the far field)
  bool batch = false;

  // cached work lists and device copies of layouts (keyed by content)
  std::map<uint64_t, std::unique_ptr<ItemPlan>> plans;
  std::map<uint64_t, std::unique_ptr<DevBuf<int4>>> layouts;
  const int4* lay_dev(const SysLayout& L);  // {geo_off, n, vec_off, chg_off} per system

  // solution state
  DevBuf<double> u;  // n_rhs * 2n
  DevBuf<double> b;  // n_rhs * 2n
  DevBuf<double> e_dev;
  DevBuf<double> phi_reac;
  bool have_solution = false;
  bipb_medium solved_medium{0, 0, 0};

  int mv32_variant = kFirstSymVariant + 2;  // FP32 mat-vec variant (the autotuner may change it)
  bool sym_pairs = true;  // FP64 / double-float mat-vecs visit unordered pairs once (sym.cu)
  bool tcx_enabled = true;  // the double-float multi-RHS mat-vec on the tensor cores (mrhs_df.cu)
  GmresWork* gw = nullptr;
  // far-field mat-vec: parameters (bipb_treecode) and the built operator
  double far_theta = 0.5;
  int far_degree = 6, far_leaf = 256;
  std::unique_ptr<FarField> far;
  KernelTimer timer;
  uint64_t alloc_gen = 0;  // bumped whenever a scratch buffer moves (recorded graphs go stale)
  long long launches = 0;           // kernels launched on this handle (graph replays included)
  bool recording = false;           // a CUDA graph is being recorded
  long long recorded_launches = 0;  // kernels in the graph being recorded

  template <typename T>
  void grow(DevBuf<T>& buf, size_t count) {
    if (buf.ensure(count, stream)) ++alloc_gen;
  }
};

Surface* checked(bipb_surface s);
void set_last_error(const std::string& msg);  // the message bipb_last_error() returns on this thread

// Brackets one kernel launch with timing events when the timer is on.
struct TimedLaunch {
  Surface* s;
  EventPair ev{0, nullptr, nullptr};
  TimedLaunch(Surface* sf, int kind) : s(sf) {
    if (!s->timer.on) return;
    ev = EventPair{kind, s->timer.get(), s->timer.get()};
    // while a graph is recorded, only an "external" record becomes a node
    // that stamps the event on every replay
    BIPB_CUDA(cudaEventRecordWithFlags(ev.a, s->stream, s->recording ? cudaEventRecordExternal : 0));
  }
  ~TimedLaunch() {
    if (!ev.a) return;
    if (cudaEventRecordWithFlags(ev.b, s->stream, s->recording ? cudaEventRecordExternal : 0) != cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    if (s->timer.capture)
      s->timer.capture->push_back(ev);
    else
      s->timer.pending.push_back(ev);
  }
};

// ---- kernels.cu: batched passes on device memory, all on s->stream ----
// Vectors are batched: system k's 2 n[k] values start at L.vec_off[k].
// y = A u or A^T u for every system; skip (device ints, stride skip_stride,
// one per system, or nullptr) makes the kernels skip systems whose flag is set.
void matvec(Surface* s, const SysLayout& L, const bipb_medium& m, int precision, bool transpose, const double* u,
            double* y, const int* skip, int skip_stride);
// Time every FP32 mat-vec variant on layout L (reps launches each) and keep
// the fastest; returns its index and its time per mat-vec in best_ms.
int autotune_matvec32(Surface* s, const SysLayout& L, const bipb_medium& m, int reps, double* best_ms);
// ---- sym.cu: mat-vecs visiting every unordered pair once; false when the
// layout is too large for the symmetric work list, or 0 < kappa < 1e-6
// (nothing launched then)
bool matvec_sym32(Surface* s, const SysLayout& L, const PairConst<float>& c, double kappa, bool transpose,
                  int variant, const double* u, double* y, double dphi, double dpsi, const int* skip,
                  int skip_stride);
bool matvec_sym64(Surface* s, const SysLayout& L, const PairConst<double>& c, double kappa, bool transpose,
                  const double* u, double* y, double dphi, double dpsi, const int* skip, int skip_stride);
bool matvec_sym_df(Surface* s, const SysLayout& L, const DFConst& c, double kappa, bool transpose, const double* u,
                   double* y, double dphi, double dpsi, const int* skip, int skip_stride);
// y = A u (or A^T u) for right-hand sides of one surface by the far-field treecode (tree.cu)
void matvec_tree(Surface* s, const SysLayout& L, const PairConst<float>& c, bool transpose, const double* u, double* y,
                 double dphi, double dpsi, const int* skip, int skip_stride);
// the far-field operator of the handle's parameters (built on first use; synchronises then)
FarField* far_field(Surface* s);
// y = A u (or A^T u) for right-hand sides of one surface with the split-FP16
// tensor-core kernel (mrhs_tc.cu)
void matvec_tc(Surface* s, const SysLayout& L, const PairConst<float>& c, bool transpose, const double* u, double* y,
               double dphi, double dpsi, const int* skip, int skip_stride);
// y = A u for right-hand sides of one surface, double-float arithmetic, kernel
// blocks shared by 16 right-hand sides (mrhs_df.cu)
void matvec_df_mrhs(Surface* s, const SysLayout& L, const DFConst& c, bool transpose, const double* u, double* y,
                    double dphi, double dpsi, const int* skip, int skip_stride);
// FP64 reduction of FP64 per-split partials (kernels.cu), tab[k] = {n, splits, offset, 0}
void launch_reduce_matvec64(Surface* s, const SysLayout& L, const int4* tab, const double* part, const double* u,
                            double* y, double dphi, double dpsi, const int* skip, int skip_stride);
// FP64 reduction of FP32 per-split partials (kernels.cu), tab[k] = {n, splits, offset, 0}
void launch_reduce_matvec32(Surface* s, const SysLayout& L, const int4* tab, const float* part, const double* u,
                            double* y, double dphi, double dpsi, const int* skip, int skip_stride);
// throws if a tensor-core kernel reported a timed-out wait since the last check (synchronises)
void check_tc_error(Surface* s);
// b = [S1; S2] of every system
void source_pass(Surface* s, const SysLayout& L, const bipb_medium& m, double* b);
// reaction potential at every charge (internal units, at chg_off) and E per system (kcal/mol)
void reaction_pass(Surface* s, const SysLayout& L, const bipb_medium& m, const double* u, double* phi_reac,
                   double* e_out);
// energy row c of every system: E = 1/2 c.u
// Potential at n_pts points (device records: pts one (p, 0) per point, pts2 two,
// (p, 0) and a zero normal) for every system, internal units, into out[k n_pts + q]:
// Eq. eq_inside when inside (with S1 of the system's charges), else the
// exterior representation (Eq. eqbim_2).
void potential_pass(Surface* s, const SysLayout& L, const bipb_medium& m, const double* u, bool inside,
                    int n_pts, const double4_32a* pts, const double4_32a* pts2, double* out);
// part[k * blocks + b]: block sums of sum_{c != l} q_c q_l / |y_c - y_l| of system k;
// tab[k] = {0, 0, nc, chg_off}.
void coulomb_pass(Surface* s, const SysLayout& L, const int4* tab, double* part, int* blocks);
void energy_row_pass(Surface* s, const SysLayout& L, const bipb_medium& m, double* c);
// dE/dq (per charge) and dE/dy (3 per charge), internal units, from u and the adjoint lam
void grad_pass(Surface* s, const SysLayout& L, const bipb_medium& m, const double* u, const double* lam, double* dq,
               double* dy);

// ---- gmres.cu ----
struct SolveResult {
  int converged = 0, iters = 0, refine_steps = 0, matvecs64 = 0, matvecs32 = 0;
  double rel_residual = 0.0;
};
// Solve op(A_k) x_k = rhs_k for every system of L (batched vectors); x holds
// the initial guess (zero if !warm) and receives the solutions.  op = A or A^T.
std::vector<SolveResult> gmres_solve(Surface* s, const SysLayout& L, const bipb_medium& m,
                                     const bipb_solve_params& p, bool transpose, const double* rhs, double* x,
                                     bool warm);
void gmres_free(Surface* s);

}  // namespace bipb
