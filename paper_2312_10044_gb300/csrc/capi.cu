// The C ABI of libbipb (declared in include/bipb.h): handles, validation,
// and the solve / energy / potential / gradient drivers.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_set>

#include "internal.cuh"

namespace bipb {

namespace {

constexpr uint64_t kMagic = 0x62697062534652ull;  // "bipbSFR"
thread_local std::string g_last_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Orders the handle's private stream after the caller's stream on entry and
// the caller's stream after the private one on exit.
struct StreamJoin {
  Surface* s;
  explicit StreamJoin(Surface* sf) : s(sf) {
    BIPB_CUDA(cudaEventRecord(s->ev_in, s->user_stream));
    BIPB_CUDA(cudaStreamWaitEvent(s->stream, s->ev_in, 0));
  }
  ~StreamJoin() {
    if (cudaEventRecord(s->ev_out, s->stream) == cudaSuccess) cudaStreamWaitEvent(s->user_stream, s->ev_out, 0);
  }
};

template <class F>
bipb_status guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return BIPB_OK;
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.st;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return BIPB_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return BIPB_ERR_CUDA;
  }
}

bool finite3(const double* p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }


void validate_medium(const bipb_medium* m) {
  BIPB_REQUIRE(m != nullptr, "medium is NULL");
  BIPB_REQUIRE(std::isfinite(m->eps_in) && m->eps_in > 0, "eps_in must be finite and > 0");
  BIPB_REQUIRE(std::isfinite(m->eps_out) && m->eps_out > 0, "eps_out must be finite and > 0");
  BIPB_REQUIRE(std::isfinite(m->kappa) && m->kappa >= 0, "kappa must be finite and >= 0");
}

void validate_params(const bipb_solve_params* p) {
  BIPB_REQUIRE(p != nullptr, "params is NULL");
  validate_medium(&p->medium);
  BIPB_REQUIRE(std::isfinite(p->tol) && p->tol > 0 && p->tol < 1, "tol must lie in (0, 1)");
  BIPB_REQUIRE(p->restart >= 0 && p->restart <= kMaxRestart, "restart must lie in [1, 200] (0 = 10)");
  BIPB_REQUIRE(p->max_iter >= 0, "max_iter must be >= 0 (0 = 1000)");
  BIPB_REQUIRE(p->precision == BIPB_FP64 || p->precision == BIPB_MIXED || p->precision == BIPB_DF64 ||
                   p->precision == BIPB_MIXED_DF64 || p->precision == BIPB_MIXED_TENSOR ||
                   p->precision == BIPB_MIXED_TREE,
               "precision must be FP64, MIXED, DF64, MIXED_DF64, MIXED_TENSOR or MIXED_TREE");
  BIPB_REQUIRE(p->inner_max_iter >= 0, "inner_max_iter must be >= 0");
  BIPB_REQUIRE(std::isfinite(p->inner_tol) && p->inner_tol >= 0 && p->inner_tol < 1, "inner_tol must lie in [0, 1)");
  BIPB_REQUIRE(p->precond == BIPB_PRECOND_NONE || p->precond == BIPB_PRECOND_SELF, "unknown precond");
  BIPB_REQUIRE(p->reserved == 0, "reserved must be 0");
}

__device__ __forceinline__ uint64_t dev_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint32_t dev_bits(float v) { return __float_as_uint(v == 0.0f ? 0.0f : v); }

// Charge records (y - centre, q) of n_rhs configurations from device arrays,
// with the checks bipb_charges_set makes on the host: every value finite, and
// no charge on a centroid (the centroid with the same FP32 point, found in the
// surface's hash table, compared in FP64).  A failed check sets *err.
__global__ void k_charges_dev(int64_t nc, int n_rhs, int n_pos_sets, const double* __restrict__ pos,
                              const double* __restrict__ q, double cx, double cy, double cz,
                              const int32_t* __restrict__ slot, uint64_t mask, const double4_32a* __restrict__ tgt64,
                              double4_32a* __restrict__ rec, int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc * n_rhs) return;
  const int64_t r = i / nc, k = i % nc;
  const double* P = pos + 3 * ((n_pos_sets == 1 ? 0 : r) * nc + k);
  const double p0 = P[0] - cx, p1 = P[1] - cy, p2 = P[2] - cz, qq = q[i];
  bool ok = isfinite(P[0]) && isfinite(P[1]) && isfinite(P[2]) && isfinite(qq);
  if (ok) {
    const float f0 = (float)p0, f1 = (float)p1, f2 = (float)p2;
    const uint64_t key = ((uint64_t)dev_bits(f0) << 32 | dev_bits(f1)) ^ dev_mix(dev_bits(f2));
    uint64_t h = dev_mix(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
      const int32_t j = slot[h];
      if (j < 0) break;
      const double4_32a g = tgt64[2 * (size_t)j];
      if (dev_bits((float)g.x) == dev_bits(f0) && dev_bits((float)g.y) == dev_bits(f1) &&
          dev_bits((float)g.z) == dev_bits(f2)) {
        ok = !(g.x == p0 && g.y == p1 && g.z == p2);
        break;
      }
    }
  }
  if (!ok) atomicOr(err, 1);
  rec[i] = make_double4_32a(p0, p1, p2, qq);
}

__global__ void k_scale(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i];
}

}  // namespace

// Live handles: a handle is dereferenced only after it is found here, so a
// destroyed or made-up handle is rejected instead of being read.
std::mutex g_live_mu;
std::unordered_set<const Surface*> g_live;

void register_handle(const Surface* s) {
  std::lock_guard<std::mutex> lk(g_live_mu);
  g_live.insert(s);
}
bool unregister_handle(const Surface* s) {
  std::lock_guard<std::mutex> lk(g_live_mu);
  return g_live.erase(s) == 1;
}
bool is_live(const Surface* s) {
  std::lock_guard<std::mutex> lk(g_live_mu);
  return g_live.count(s) == 1;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }

Surface* checked(bipb_surface h) {
  Surface* s = reinterpret_cast<Surface*>(h);
  if (s == nullptr || !is_live(s) || s->magic != kMagic)
    throw Error(BIPB_ERR_STATE, "invalid or destroyed surface handle");
  return s;
}

}  // namespace bipb

using namespace bipb;

// The stream-ordered pool of a device keeps up to 4 GiB of freed memory for
// reuse (this process only; the driver default returns it at every
// synchronisation).
namespace bipb {
void keep_pool_memory(int device) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lock(mu);
  if (std::find(done.begin(), done.end(), device) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = 4ull << 30;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) (void)cudaGetLastError();
  } else {
    (void)cudaGetLastError();
  }
  done.push_back(device);
}
}  // namespace bipb

extern "C" {

const char* bipb_version(void) { return "bipb 0.1 (sm_103a)"; }

const char* bipb_last_error(void) { return g_last_error.c_str(); }

const char* bipb_status_string(bipb_status st) {
  switch (st) {
    case BIPB_OK: return "ok";
    case BIPB_ERR_INVALID_ARG: return "invalid argument";
    case BIPB_ERR_CUDA: return "CUDA error";
    case BIPB_ERR_OOM: return "out of device memory";
    case BIPB_ERR_NOT_CONVERGED: return "not converged";
    case BIPB_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

int64_t bipb_surface_size(bipb_surface h) {
  Surface* s = reinterpret_cast<Surface*>(h);
  return (s && is_live(s)) ? s->n : 0;
}

namespace {

struct PartIn {
  int64_t n;
  const double *c, *nrm, *area;
};

// Validate one surface and append it (centred on its own mean centroid) to
// the host geometry arrays.
void add_part(Surface* s, const PartIn& P, std::vector<double4_32a>& tgt, std::vector<float4>& tgt32) {
  BIPB_REQUIRE(P.n >= 2, "need at least 2 triangles per surface");
  BIPB_REQUIRE(P.c && P.nrm && P.area, "NULL input array");
  double c[3] = {0, 0, 0};
  std::vector<double> inv_len((size_t)P.n);
  for (int64_t i = 0; i < P.n; ++i) {
    BIPB_REQUIRE(finite3(P.c + 3 * i), "non-finite centroid");
    BIPB_REQUIRE(finite3(P.nrm + 3 * i), "non-finite normal");
    BIPB_REQUIRE(std::isfinite(P.area[i]) && P.area[i] > 0, "areas must be finite and > 0");
    const double* v = P.nrm + 3 * i;
    double len = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    BIPB_REQUIRE(std::fabs(len - 1.0) <= 1e-6, "normals must have unit length (within 1e-6)");
    inv_len[i] = 1.0 / len;
    for (int k = 0; k < 3; ++k) c[k] += P.c[3 * i + k];
  }
  for (int k = 0; k < 3; ++k) c[k] /= (double)P.n;
  // centred copies (FP64 and FP32 records), and the check for duplicates (in
  // FP32, then FP64 on a hit); the set is kept to reject charges on a centroid
  CentroidSet cs;
  cs.d.resize(3 * (size_t)P.n);
  cs.f.resize(3 * (size_t)P.n);
  cs.reserve((size_t)P.n);
  const size_t base = tgt.size();
  tgt.resize(base + 2 * (size_t)P.n);
  tgt32.resize(base + 2 * (size_t)P.n);
  for (int64_t i = 0; i < P.n; ++i) {
    double* d = &cs.d[3 * i];
    float* f = &cs.f[3 * i];
    for (int k = 0; k < 3; ++k) {
      d[k] = P.c[3 * i + k] - c[k];
      f[k] = (float)d[k];
    }
    const int32_t j = cs.insert((int32_t)i);
    if (j >= 0) {
      const bool same64 = cs.d[3 * j] == d[0] && cs.d[3 * j + 1] == d[1] && cs.d[3 * j + 2] == d[2];
      throw Error(BIPB_ERR_INVALID_ARG,
                  same64 ? "two centroids coincide" : "two centroids coincide after rounding to FP32");
    }
    const double* v = P.nrm + 3 * i;
    const double nx = v[0] * inv_len[i], ny = v[1] * inv_len[i], nz = v[2] * inv_len[i];
    tgt[base + 2 * i] = make_double4_32a(d[0], d[1], d[2], P.area[i]);
    tgt[base + 2 * i + 1] = make_double4_32a(nx, ny, nz, 0.0);
    tgt32[base + 2 * i] = make_float4(f[0], f[1], f[2], (float)P.area[i]);
    tgt32[base + 2 * i + 1] = make_float4((float)nx, (float)ny, (float)nz, 0.f);
  }
  s->part_off.push_back((int)s->n);
  s->part_n.push_back((int)P.n);
  for (int k = 0; k < 3; ++k) s->part_center.push_back(c[k]);
  s->part_keys.push_back(std::move(cs));
  s->n += P.n;
}

// 2^(j/1024) for j < 1024 as df64 (hi, lo) pairs, two per float4: the table
// of the df64 exp (df64.cuh)
const std::vector<float4>& exp_table() {
  static const std::vector<float4> t = [] {
    std::vector<float4> v(kExpTab / 2);
    auto hi = [](int j) { return (float)std::exp2(j / (double)kExpTab); };
    auto lo = [](int j) {
      const double x = std::exp2(j / (double)kExpTab);
      return (float)(x - (double)(float)x);
    };
    for (int i = 0; i < kExpTab / 2; ++i) v[i] = make_float4(hi(2 * i), lo(2 * i), hi(2 * i + 1), lo(2 * i + 1));
    return v;
  }();
  return t;
}

bipb_surface create_surface(const std::vector<PartIn>& parts, void* cuda_stream, bool batch) {
  auto* s = new Surface();
  try {
    std::vector<double4_32a> tgt;
    std::vector<float4> tgt32;
    int64_t total = 0;
    for (auto& P : parts) total += std::max<int64_t>(P.n, 0);
    BIPB_REQUIRE(total <= (int64_t)1 << 28, "at most 2^28 triangles");
    tgt.reserve(2 * total);
    tgt32.reserve(2 * total);
    for (auto& P : parts) add_part(s, P, tgt, tgt32);
    s->batch = batch;
    if (!batch) s->raw_centroids.assign(parts[0].c, parts[0].c + 3 * parts[0].n);
    int dev = 0;
    BIPB_CUDA(cudaGetDevice(&dev));
    s->device = dev;
    BIPB_CUDA(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev));
    s->user_stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    BIPB_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    BIPB_CUDA(cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming));
    BIPB_CUDA(cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming));
    keep_pool_memory(dev);
    s->tgt64.ensure(tgt.size(), s->stream);
    s->tgt32.ensure(tgt32.size(), s->stream);
    const std::vector<float4>& et = exp_table();
    s->exptab.ensure(et.size(), s->stream);
    BIPB_CUDA(cudaMemcpyAsync(s->exptab.p, et.data(), et.size() * sizeof(float4), cudaMemcpyHostToDevice,
                              s->stream));
    BIPB_CUDA(cudaMemcpyAsync(s->tgt64.p, tgt.data(), tgt.size() * sizeof(double4_32a), cudaMemcpyHostToDevice,
                              s->stream));
    BIPB_CUDA(cudaMemcpyAsync(s->tgt32.p, tgt32.data(), tgt32.size() * sizeof(float4), cudaMemcpyHostToDevice,
                              s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    s->magic = kMagic;
  } catch (...) {
    cudaStream_t st = s->stream;
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    delete s;  // its buffers go back to the pool on its stream
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    throw;
  }
  register_handle(s);
  return reinterpret_cast<bipb_surface>(s);
}

// Charge records of one system, centred like its surface; rejects charges on
// a centroid (lookup in the surface's set of centred centroids).
void append_charges(Surface* s, int part, int64_t nc, const double* pos, const double* q,
                    std::vector<double4_32a>& rec) {
  const double* c = &s->part_center[3 * part];
  const auto& keys = s->part_keys[part];
  for (int64_t k = 0; k < nc; ++k) {
    BIPB_REQUIRE(finite3(pos + 3 * k), "non-finite charge position");
    BIPB_REQUIRE(std::isfinite(q[k]), "non-finite charge");
    double p[3] = {pos[3 * k] - c[0], pos[3 * k + 1] - c[1], pos[3 * k + 2] - c[2]};
    const float pf[3] = {(float)p[0], (float)p[1], (float)p[2]};
    const int32_t j = keys.find(pf);  // the only centroid that can equal p in FP64
    BIPB_REQUIRE(j < 0 || !(keys.d[3 * j] == p[0] && keys.d[3 * j + 1] == p[1] && keys.d[3 * j + 2] == p[2]),
                 "a charge sits on a centroid");
    rec.push_back(make_double4_32a(p[0], p[1], p[2], q[k]));
  }
}

void store_charges(Surface* s, const std::vector<double4_32a>& rec, SysLayout lay) {
  s->grow(s->chg, rec.size());
  BIPB_CUDA(cudaMemcpyAsync(s->chg.p, rec.data(), rec.size() * sizeof(double4_32a), cudaMemcpyHostToDevice,
                            s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  s->lay = std::move(lay);
  s->n_rhs = s->lay.K;
  s->have_solution = false;
}

// Layout of n_vec vectors for the device mat-vec entry point: replicas of a
// single surface, or (n_vec = 1) the surfaces of a batch handle.
SysLayout matvec_layout(Surface* s, int n_vec) {
  std::vector<int> go, n, co, nc;
  if (s->batch) {
    for (size_t k = 0; k < s->part_n.size(); ++k) go.push_back(s->part_off[k]), n.push_back(s->part_n[k]);
  } else {
    for (int v = 0; v < n_vec; ++v) go.push_back(0), n.push_back((int)s->n);
  }
  co.assign(go.size(), 0);
  nc.assign(go.size(), 0);
  return make_layout(go, n, co, nc);
}

// Charges passed on the device are checked on the device; the first call that
// uses them reads the result (and forgets the charges if a check failed).
void check_device_charges(Surface* s) {
  if (!s->chg_check_pending) return;
  int h = 0;
  BIPB_CUDA(cudaMemcpyAsync(&h, s->chg_err.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  s->chg_check_pending = false;
  if (h) {
    s->n_rhs = 0;
    throw Error(BIPB_ERR_INVALID_ARG, "bipb_charges_set_dev: a charge position or value is not finite, or a "
                                      "charge sits on a centroid");
  }
}

void require_charges(Surface* s) {
  BIPB_REQUIRE(s->n_rhs > 0, "no charges set");
  check_device_charges(s);
}



}  // namespace

bipb_status bipb_surface_create(int64_t n, const double* centroids, const double* normals, const double* areas,
                                void* cuda_stream, bipb_surface* out) {
  return guarded([&] {
    BIPB_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    BIPB_REQUIRE(n >= 2, "need at least 2 triangles");
    BIPB_REQUIRE(n <= (int64_t)1 << 28, "at most 2^28 triangles");
    *out = create_surface({PartIn{n, centroids, normals, areas}}, cuda_stream, false);
  });
}

bipb_status bipb_surface_create_batch(int n_surf, const int64_t* n_tri, const double* const* centroids,
                                      const double* const* normals, const double* const* areas, void* cuda_stream,
                                      bipb_surface* out) {
  return guarded([&] {
    BIPB_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    BIPB_REQUIRE(n_surf >= 1 && n_surf <= 4096, "n_surf must lie in [1, 4096]");
    BIPB_REQUIRE(n_tri && centroids && normals && areas, "NULL input array");
    std::vector<PartIn> parts;
    for (int k = 0; k < n_surf; ++k) parts.push_back(PartIn{n_tri[k], centroids[k], normals[k], areas[k]});
    *out = create_surface(parts, cuda_stream, true);
  });
}


bipb_status bipb_surface_destroy(bipb_surface h) {
  return guarded([&] {
    Surface* s = checked(h);
    if (!unregister_handle(s)) throw Error(BIPB_ERR_STATE, "invalid or destroyed surface handle");
    DeviceGuard dg(s->device);
    cudaStreamSynchronize(s->stream);
    gmres_free(s);
    s->magic = 0;
    cudaEventDestroy(s->ev_in);
    cudaEventDestroy(s->ev_out);
    cudaStream_t st = s->stream;
    delete s;  // its buffers go back to the pool on its stream
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  });
}

bipb_status bipb_charges_set(bipb_surface h, int64_t nc, const double* pos, int n_pos_sets, int n_rhs,
                             const double* q) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(!s->batch, "a batch handle takes its charges through bipb_charges_set_batch");
    BIPB_REQUIRE(nc >= 1 && nc <= (int64_t)1 << 26, "nc must lie in [1, 2^26]");
    BIPB_REQUIRE(n_rhs >= 1 && n_rhs <= 4096, "n_rhs must lie in [1, 4096]");
    BIPB_REQUIRE(n_pos_sets == 1 || n_pos_sets == n_rhs, "n_pos_sets must be 1 or n_rhs");
    BIPB_REQUIRE(pos && q, "NULL input array");
    BIPB_REQUIRE((int64_t)n_rhs * nc <= (int64_t)1 << 28, "too many charges in total");
    DeviceGuard dg(s->device);
    std::vector<double4_32a> rec;
    rec.reserve((size_t)n_rhs * nc);
    std::vector<int> go(n_rhs, 0), n(n_rhs, (int)s->n), co(n_rhs), ncv(n_rhs, (int)nc);
    for (int r = 0; r < n_rhs; ++r) {
      co[r] = (int)(r * nc);
      append_charges(s, 0, nc, pos + (size_t)(n_pos_sets == 1 ? 0 : r) * nc * 3, q + (size_t)r * nc, rec);
    }
    s->nc = nc;
    s->n_pos_sets = n_pos_sets;
    store_charges(s, rec, make_layout(go, n, co, ncv));
  });
}

bipb_status bipb_charges_set_dev(bipb_surface h, int64_t nc, const double* pos, int n_pos_sets, int n_rhs,
                                 const double* q) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(!s->batch, "a batch handle takes its charges through bipb_charges_set_batch");
    BIPB_REQUIRE(nc >= 1 && nc <= (int64_t)1 << 26, "nc must lie in [1, 2^26]");
    BIPB_REQUIRE(n_rhs >= 1 && n_rhs <= 4096, "n_rhs must lie in [1, 4096]");
    BIPB_REQUIRE(n_pos_sets == 1 || n_pos_sets == n_rhs, "n_pos_sets must be 1 or n_rhs");
    BIPB_REQUIRE(pos && q, "NULL input array");
    BIPB_REQUIRE((int64_t)n_rhs * nc <= (int64_t)1 << 28, "too many charges in total");
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    const CentroidSet& keys = s->part_keys[0];
    if (s->key_slots.cap == 0) {
      s->key_slots.ensure(keys.slot.size(), s->stream);
      BIPB_CUDA(cudaMemcpyAsync(s->key_slots.p, keys.slot.data(), keys.slot.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, s->stream));
      s->chg_err.ensure(1, s->stream);
      ++s->alloc_gen;
    }
    const int64_t total = (int64_t)n_rhs * nc;
    s->grow(s->chg, (size_t)total);
    BIPB_CUDA(cudaMemsetAsync(s->chg_err.p, 0, sizeof(int), s->stream));
    const double* c = &s->part_center[0];
    k_charges_dev<<<(unsigned)((total + 255) / 256), 256, 0, s->stream>>>(
        nc, n_rhs, n_pos_sets, pos, q, c[0], c[1], c[2], s->key_slots.p, keys.mask, s->tgt64.p, s->chg.p,
        s->chg_err.p);
    BIPB_LAUNCHED(s);
    std::vector<int> go(n_rhs, 0), n(n_rhs, (int)s->n), co(n_rhs), ncv(n_rhs, (int)nc);
    for (int r = 0; r < n_rhs; ++r) co[r] = (int)(r * nc);
    s->nc = nc;
    s->n_pos_sets = n_pos_sets;
    s->lay = make_layout(go, n, co, ncv);
    s->n_rhs = s->lay.K;
    s->have_solution = false;
    s->chg_check_pending = true;
  });
}

bipb_status bipb_charges_set_batch(bipb_surface h, const int64_t* nc, const double* const* pos,
                                   const double* const* q) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(s->batch, "bipb_charges_set_batch needs a batch handle");
    BIPB_REQUIRE(nc && pos && q, "NULL input array");
    const int K = (int)s->part_n.size();
    DeviceGuard dg(s->device);
    std::vector<double4_32a> rec;
    std::vector<int> co(K), ncv(K);
    for (int k = 0; k < K; ++k) {
      BIPB_REQUIRE(nc[k] >= 1 && nc[k] <= (int64_t)1 << 26, "every surface needs 1 .. 2^26 charges");
      BIPB_REQUIRE(pos[k] && q[k], "NULL charge array");
      co[k] = (int)rec.size();
      ncv[k] = (int)nc[k];
      append_charges(s, k, nc[k], pos[k], q[k], rec);
      BIPB_REQUIRE(rec.size() <= ((size_t)1 << 28), "too many charges in total");
    }
    s->nc = 0;
    s->n_pos_sets = 0;
    store_charges(s, rec, make_layout(s->part_off, s->part_n, co, ncv));
  });
}

bipb_status bipb_source(bipb_surface h, const bipb_medium* m, double* b) {
  return guarded([&] {
    Surface* s = checked(h);
    validate_medium(m);
    BIPB_REQUIRE(b != nullptr, "b is NULL");
    require_charges(s);
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    source_pass(s, s->lay, *m, b);
  });
}

bipb_status bipb_matvec(bipb_surface h, const bipb_medium* m, int precision, int transpose, int n_vec,
                        const double* u, double* y) {
  return guarded([&] {
    Surface* s = checked(h);
    validate_medium(m);
    BIPB_REQUIRE(precision == BIPB_FP64 || precision == BIPB_FP32 || precision == BIPB_DF64 ||
                     precision == BIPB_TENSOR || precision == BIPB_TREE32,
                 "precision must be FP64, FP32, DF64, TENSOR or TREE32");
    BIPB_REQUIRE(precision != BIPB_TENSOR || !s->batch, "the tensor-core mat-vec needs a single-surface handle");
    BIPB_REQUIRE(precision != BIPB_TREE32 || !s->batch, "the far-field mat-vec needs a single-surface handle");
    BIPB_REQUIRE(n_vec >= 1 && n_vec <= 4096, "n_vec must lie in [1, 4096]");
    BIPB_REQUIRE(!s->batch || n_vec == 1, "a batch handle takes one batched vector (n_vec = 1)");
    BIPB_REQUIRE(u && y, "NULL vector");
    BIPB_REQUIRE(u != y, "y must not alias u");
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    matvec(s, matvec_layout(s, n_vec), *m, precision, transpose != 0, u, y, nullptr, 0);
    if (precision == BIPB_TENSOR) check_tc_error(s);
  });
}

bipb_status bipb_reaction(bipb_surface h, const bipb_medium* m, const double* u, double* phi_reac,
                          double* e_sol) {
  return guarded([&] {
    Surface* s = checked(h);
    validate_medium(m);
    BIPB_REQUIRE(u != nullptr, "u is NULL");
    require_charges(s);
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    reaction_pass(s, s->lay, *m, u, phi_reac, e_sol);
  });
}

bipb_status bipb_solve(bipb_surface h, const bipb_solve_params* p, bipb_solve_info* info) {
  bipb_status st = BIPB_OK;
  bipb_status rc = guarded([&] {
    auto t0 = std::chrono::steady_clock::now();
    Surface* s = checked(h);
    validate_params(p);
    require_charges(s);
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    const SysLayout& L = s->lay;
    s->grow(s->u, L.len);
    s->grow(s->b, L.len);
    s->grow(s->e_dev, L.K);
    if (p->x0) {
      for (int64_t i = 0; i < L.len; ++i) BIPB_REQUIRE(std::isfinite(p->x0[i]), "non-finite x0");
      BIPB_CUDA(cudaMemcpyAsync(s->u.p, p->x0, L.len * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    }
    s->have_solution = false;
    source_pass(s, L, p->medium, s->b.p);
    BIPB_REQUIRE(p->precision != BIPB_MIXED_TENSOR || !s->batch, "MIXED_TENSOR needs a single-surface handle");
    BIPB_REQUIRE(p->precision != BIPB_MIXED_TREE || !s->batch, "MIXED_TREE needs a single-surface handle");
    std::vector<SolveResult> res = gmres_solve(s, L, p->medium, *p, false, s->b.p, s->u.p, p->x0 != nullptr);
    if (p->precision == BIPB_MIXED_TENSOR) check_tc_error(s);
    reaction_pass(s, L, p->medium, s->u.p, nullptr, s->e_dev.p);
    for (auto& r : res)
      if (!r.converged) st = BIPB_ERR_NOT_CONVERGED;
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    s->have_solution = true;
    s->solved_medium = p->medium;
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
      for (int r = 0; r < L.K; ++r) {
        info[r].converged = res[r].converged;
        info[r].iters = res[r].iters;
        info[r].refine_steps = res[r].refine_steps;
        info[r].matvecs64 = res[r].matvecs64;
        info[r].matvecs32 = res[r].matvecs32;
        info[r].reserved = 0;
        info[r].rel_residual = res[r].rel_residual;
        info[r].seconds = secs;
      }
    }
  });
  if (rc != BIPB_OK) return rc;
  if (st != BIPB_OK) g_last_error = "at least one right-hand side did not reach tol within max_iter";
  return st;
}

bipb_status bipb_energy(bipb_surface h, double* e_sol) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(e_sol != nullptr, "e_sol is NULL");
    if (!s->have_solution) throw Error(BIPB_ERR_STATE, "bipb_solve has not run since the charges were set");
    DeviceGuard dg(s->device);
    BIPB_CUDA(cudaMemcpyAsync(e_sol, s->e_dev.p, s->lay.K * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
  });
}

bipb_status bipb_energy_dev(bipb_surface h, double* e_sol) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(e_sol != nullptr, "e_sol is NULL");
    if (!s->have_solution) throw Error(BIPB_ERR_STATE, "bipb_solve has not run since the charges were set");
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    BIPB_CUDA(cudaMemcpyAsync(e_sol, s->e_dev.p, s->lay.K * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  });
}

bipb_status bipb_surface_potential(bipb_surface h, double* phi, double* dphi_dn) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(phi != nullptr, "phi is NULL");
    if (!s->have_solution) throw Error(BIPB_ERR_STATE, "bipb_solve has not run since the charges were set");
    DeviceGuard dg(s->device);
    const SysLayout& L = s->lay;
    std::vector<double> u(L.len);
    BIPB_CUDA(cudaMemcpyAsync(u.data(), s->u.p, u.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    size_t out = 0;
    for (int k = 0; k < L.K; ++k) {
      const size_t n = L.n[k], v = L.vec_off[k];
      for (size_t i = 0; i < n; ++i) {
        phi[out + i] = kKcal * u[v + i];
        if (dphi_dn) dphi_dn[out + i] = kKcal * u[v + n + i];
      }
      out += n;
    }
  });
}

bipb_status bipb_potential_at(bipb_surface h, int region, int64_t n_pts, const double* pts, double* phi) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(region == BIPB_REGION_INSIDE || region == BIPB_REGION_OUTSIDE, "unknown region");
    BIPB_REQUIRE(n_pts >= 0 && n_pts <= ((int64_t)1 << 24), "n_pts must be in [0, 2^24]");
    BIPB_REQUIRE(n_pts == 0 || (pts != nullptr && phi != nullptr), "pts or phi is NULL");
    BIPB_REQUIRE(!s->batch, "bipb_potential_at takes single-surface handles");
    if (!s->have_solution) throw Error(BIPB_ERR_STATE, "bipb_solve has not run since the charges were set");
    if (n_pts == 0) return;
    const SysLayout& L = s->lay;
    // the points in the frame of the surface's centred copies
    const double* c = &s->part_center[0];
    std::vector<double4_32a> p1((size_t)n_pts), p2((size_t)2 * n_pts);
    for (int64_t i = 0; i < n_pts; ++i) {
      double d[3];
      for (int k = 0; k < 3; ++k) {
        BIPB_REQUIRE(std::isfinite(pts[3 * i + k]), "non-finite point");
        d[k] = pts[3 * i + k] - c[k];
      }
      p1[i] = double4_32a{d[0], d[1], d[2], 0.0};
      p2[2 * i] = p1[i];
      p2[2 * i + 1] = double4_32a{0.0, 0.0, 0.0, 0.0};
    }
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    s->grow(s->pts, (size_t)n_pts);
    s->grow(s->pts2, (size_t)2 * n_pts);
    s->grow(s->pot, (size_t)L.K * n_pts);
    BIPB_CUDA(cudaMemcpyAsync(s->pts.p, p1.data(), p1.size() * sizeof(double4_32a), cudaMemcpyHostToDevice,
                              s->stream));
    BIPB_CUDA(cudaMemcpyAsync(s->pts2.p, p2.data(), p2.size() * sizeof(double4_32a), cudaMemcpyHostToDevice,
                              s->stream));
    potential_pass(s, L, s->solved_medium, s->u.p, region == BIPB_REGION_INSIDE, (int)n_pts, s->pts.p, s->pts2.p,
                   s->pot.p);
    BIPB_CUDA(cudaMemcpyAsync(phi, s->pot.p, (size_t)L.K * n_pts * sizeof(double), cudaMemcpyDeviceToHost,
                              s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < (int64_t)L.K * n_pts; ++i) phi[i] *= kKcal;
  });
}

bipb_status bipb_energy_free(bipb_surface h, double* e_free, double* e_coul) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(e_free || e_coul, "both outputs are NULL");
    if (!s->have_solution) throw Error(BIPB_ERR_STATE, "bipb_solve has not run since the charges were set");
    const SysLayout& L = s->lay;
    std::vector<int4> tab(L.K);
    for (int k = 0; k < L.K; ++k) tab[k] = make_int4(0, 0, L.nc[k], L.chg_off[k]);
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    s->grow(s->coul_tab, (size_t)L.K);
    BIPB_CUDA(cudaMemcpyAsync(s->coul_tab.p, tab.data(), tab.size() * sizeof(int4), cudaMemcpyHostToDevice,
                              s->stream));
    int nc_max = 1;
    for (int k = 0; k < L.K; ++k) nc_max = std::max(nc_max, L.nc[k]);
    s->grow(s->coul, (size_t)L.K * ((nc_max + 255) / 256));
    int blocks = 0;
    coulomb_pass(s, L, s->coul_tab.p, s->coul.p, &blocks);
    std::vector<double> part((size_t)L.K * blocks), es(L.K);
    BIPB_CUDA(cudaMemcpyAsync(part.data(), s->coul.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                              s->stream));
    BIPB_CUDA(cudaMemcpyAsync(es.data(), s->e_dev.p, es.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    for (int k = 0; k < L.K; ++k) {
      double acc = 0.0;
      for (int b = 0; b < blocks; ++b) acc += part[(size_t)k * blocks + b];
      // 1/2 (1/eps_in) sum_{c != l} q_c q_l / (4 pi r) in internal units, times 4 pi 332.0716
      const double ec = 0.5 * 332.0716 / s->solved_medium.eps_in * acc;
      BIPB_REQUIRE(std::isfinite(ec), "two charges coincide: their Coulomb energy is infinite");
      if (e_coul) e_coul[k] = ec;
      if (e_free) e_free[k] = es[k] + ec;
    }
  });
}

namespace {
// Adjoint solve and gradient pass into device buffers dq (per charge) and dy
// (3 per charge), internal units; returns BIPB_ERR_NOT_CONVERGED if an
// adjoint solve missed tol.
bipb_status energy_grad_device(Surface* s, const bipb_solve_params* p, DevBuf<double>& dq, DevBuf<double>& dy,
                               size_t* n_chg_out) {
  validate_params(p);
  if (!s->have_solution) throw Error(BIPB_ERR_STATE, "bipb_solve has not run since the charges were set");
  const bipb_medium& m = s->solved_medium;
  BIPB_REQUIRE(p->medium.eps_in == m.eps_in && p->medium.eps_out == m.eps_out && p->medium.kappa == m.kappa,
               "params.medium differs from the medium of the last solve");
  const SysLayout& L = s->lay;
  size_t n_chg = 0;
  for (int k = 0; k < L.K; ++k) n_chg += L.nc[k];
  DevBuf<double> c, lam;
  c.ensure(L.len, s->stream);
  lam.ensure(L.len, s->stream);
  dq.ensure(n_chg, s->stream);
  dy.ensure(3 * n_chg, s->stream);
  bipb_solve_params pa = *p;
  pa.x0 = nullptr;
  energy_row_pass(s, L, m, c.p);
  std::vector<SolveResult> res = gmres_solve(s, L, m, pa, true, c.p, lam.p, false);
  bipb_status st = BIPB_OK;
  for (auto& r : res)
    if (!r.converged) st = BIPB_ERR_NOT_CONVERGED;
  grad_pass(s, L, m, s->u.p, lam.p, dq.p, dy.p);
  *n_chg_out = n_chg;
  return st;
}
}  // namespace

bipb_status bipb_energy_grad_dev(bipb_surface h, const bipb_solve_params* p, double* dE_dq, double* dE_dpos) {
  bipb_status st = BIPB_OK;
  bipb_status rc = guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(dE_dq || dE_dpos, "both outputs are NULL");
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    DevBuf<double> dq, dy;
    size_t n_chg = 0;
    st = energy_grad_device(s, p, dq, dy, &n_chg);
    if (dE_dq) {
      k_scale<<<(unsigned)((n_chg + 255) / 256), 256, 0, s->stream>>>((int64_t)n_chg, kKcal, dq.p, dE_dq);
      BIPB_LAUNCHED(s);
    }
    if (dE_dpos) {
      k_scale<<<(unsigned)((3 * n_chg + 255) / 256), 256, 0, s->stream>>>((int64_t)(3 * n_chg), kKcal, dy.p, dE_dpos);
      BIPB_LAUNCHED(s);
    }
  });
  if (rc != BIPB_OK) return rc;
  if (st != BIPB_OK) g_last_error = "an adjoint solve did not reach tol within max_iter";
  return st;
}

bipb_status bipb_energy_grad(bipb_surface h, const bipb_solve_params* p, double* dE_dq, double* dE_dpos) {
  bipb_status st = BIPB_OK;
  bipb_status rc = guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(dE_dq || dE_dpos, "both outputs are NULL");
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    DevBuf<double> dq, dy;
    size_t n_chg = 0;
    st = energy_grad_device(s, p, dq, dy, &n_chg);
    std::vector<double> hq(n_chg), hy(3 * n_chg);
    BIPB_CUDA(cudaMemcpyAsync(hq.data(), dq.p, n_chg * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    BIPB_CUDA(cudaMemcpyAsync(hy.data(), dy.p, 3 * n_chg * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    for (size_t k = 0; k < n_chg; ++k) {
      if (dE_dq) dE_dq[k] = kKcal * hq[k];
      if (dE_dpos)
        for (int a = 0; a < 3; ++a) dE_dpos[3 * k + a] = kKcal * hy[3 * k + a];
    }
  });
  if (rc != BIPB_OK) return rc;
  if (st != BIPB_OK) g_last_error = "an adjoint solve did not reach tol within max_iter";
  return st;
}

bipb_status bipb_autotune(bipb_surface h, const bipb_medium* m, int reps, int* variant, double* ms_per_matvec) {
  return guarded([&] {
    Surface* s = checked(h);
    validate_medium(m);
    BIPB_REQUIRE(reps >= 1 && reps <= 1000, "reps must lie in [1, 1000]");
    DeviceGuard dg(s->device);
    StreamJoin sj(s);
    const SysLayout L = s->n_rhs > 0 ? s->lay : matvec_layout(s, 1);
    int v = autotune_matvec32(s, L, *m, reps, ms_per_matvec);
    if (variant) *variant = v;
  });
}

bipb_status bipb_matvec_variant(bipb_surface h, int variant) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(variant >= 0 && variant < kNumMv32Variants, "unknown FP32 mat-vec variant");
    s->mv32_variant = variant;
  });
}

bipb_status bipb_symmetric_pairs(bipb_surface h, int symmetric) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(symmetric == 0 || symmetric == 1, "symmetric must be 0 or 1");
    s->sym_pairs = symmetric != 0;
  });
}

bipb_status bipb_exact_tensor_residual(bipb_surface h, int tensor) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(tensor == 0 || tensor == 1, "tensor must be 0 or 1");
    s->tcx_enabled = tensor != 0;
  });
}

bipb_status bipb_treecode(bipb_surface h, double theta, int degree, int leaf_size) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(!s->batch, "the far-field mat-vec needs a single-surface handle");
    BIPB_REQUIRE(std::isfinite(theta) && theta >= 0.0 && theta < 1.0, "theta must lie in [0, 1)");
    BIPB_REQUIRE(degree == 4 || degree == 6 || degree == 8, "degree must be 4, 6 or 8");
    BIPB_REQUIRE(leaf_size >= 32 && leaf_size <= 512, "leaf_size must lie in [32, 512]");
    s->far_theta = theta;
    s->far_degree = degree;
    s->far_leaf = leaf_size;
  });
}

bipb_status bipb_treecode_stats(bipb_surface h, int64_t* pairs, int* far_clusters, int* leaves) {
  return guarded([&] {
    Surface* s = checked(h);
    DeviceGuard dg(s->device);
    FarField* f = far_field(s);
    if (pairs) *pairs = f->pair_evals;
    if (far_clusters) *far_clusters = f->n_slots;
    if (leaves) *leaves = f->n_leaves;
  });
}

bipb_status bipb_launch_count(bipb_surface h, int64_t* launches) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(launches != nullptr, "launches is NULL");
    *launches = s->launches;
  });
}

bipb_status bipb_timer_enable(bipb_surface h, int on) {
  return guarded([&] {
    Surface* s = checked(h);
    DeviceGuard dg(s->device);
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    s->timer.collect();
    s->timer.reset();
    s->timer.on = on != 0;
  });
}

bipb_status bipb_timer_read(bipb_surface h, int kind, int64_t* launches, double* total_ms) {
  return guarded([&] {
    Surface* s = checked(h);
    BIPB_REQUIRE(kind >= 0 && kind < kTKinds, "unknown kernel kind");
    DeviceGuard dg(s->device);
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    s->timer.collect();
    if (launches) *launches = s->timer.count[kind];
    if (total_ms) *total_ms = s->timer.total_ms[kind];
  });
}

}  // extern "C"
