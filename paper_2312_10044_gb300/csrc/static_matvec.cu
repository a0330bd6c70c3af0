// bipb_matvec32_static: the FP32 mat-vec y = A u for callers that must not
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or unwelcome,
// for example a host framework whose own allocator has reserved nearly all
// device memory (a second allocator would fail or fragment it), or a
// time-critical loop (molecular dynamics, Monte Carlo) that forbids
// allocation after start-up.  Such callers cannot create a bipb_surface,
// because creating one allocates.  This entry point takes the geometry and
// the vectors as device pointers and keeps its scratch (FP32 target and
// source records, per-split partial sums, the mean centroid) in one
// statically sized device array that every GPU loading the library holds
// until the process exits.
//
// The array's name, seen from host code, is only a host-side stand-in: a
// kernel given it would fault or, where the GPU can reach host memory,
// silently read the wrong memory.  The device address is therefore looked up
// once per device with cudaGetSymbolAddress (on the first call made with
// that device current) and passed to the kernels.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace bipb {
namespace {

constexpr int64_t kStaticMaxN = 32768;  // largest surface this entry point accepts
constexpr int kSNT = 256, kSTPT = 2, kSCH = 128;
constexpr int kStaticMaxSplits = 32;
constexpr int64_t kStaticMaxPad = (kStaticMaxN + kSCH - 1) / kSCH * kSCH;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
// layout of the scratch array (byte offsets, each 256-byte aligned)
constexpr size_t kOffCenter = 0;                                                  // 4 doubles
constexpr size_t kOffTgt = align256(kOffCenter + 4 * sizeof(double));             // 2 float4 per target
constexpr size_t kOffRec = align256(kOffTgt + 2 * kStaticMaxN * sizeof(float4));  // 2 float4 per source
constexpr size_t kOffPart = align256(kOffRec + 2 * kStaticMaxPad * sizeof(float4));
constexpr size_t kStaticBytes = align256(kOffPart + (size_t)kStaticMaxSplits * 2 * kStaticMaxN * sizeof(float));

// about 10 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr double kFarS = 1.0e10;
constexpr double kInv4PiS = 1.0 / (4.0 * kPi);

// mean centroid in one block, fixed order
__global__ void k_static_center(int n, const double* __restrict__ cen, unsigned char* __restrict__ scratch) {
  __shared__ double red[3][256];
  double acc[3] = {0, 0, 0};
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int k = 0; k < 3; ++k) acc[k] += cen[3 * i + k];
  for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* c = reinterpret_cast<double*>(scratch + kOffCenter);
    for (int k = 0; k < 3; ++k) c[k] = red[k][0] / n;
  }
}

// FP32 target records (centred x, n) and forward source records
// (x, ds psi), (ds phi n, 0); zero records far away pad the last chunk.
__global__ void k_static_pack(int n, int n_pad, const double* __restrict__ cen, const double* __restrict__ nrm,
                              const double* __restrict__ area, const double* __restrict__ u,
                              unsigned char* __restrict__ scratch) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_pad) return;
  const double* c = reinterpret_cast<const double*>(scratch + kOffCenter);
  float4* tgt = reinterpret_cast<float4*>(scratch + kOffTgt);
  float4* rec = reinterpret_cast<float4*>(scratch + kOffRec);
  if (j < n) {
    float x = (float)(cen[3 * j] - c[0]), y = (float)(cen[3 * j + 1] - c[1]), z = (float)(cen[3 * j + 2] - c[2]);
    double nx = nrm[3 * j], ny = nrm[3 * j + 1], nz = nrm[3 * j + 2];
    double a = area[j], fphi = a * u[j];
    tgt[2 * j] = make_float4(x, y, z, (float)a);
    tgt[2 * j + 1] = make_float4((float)nx, (float)ny, (float)nz, 0.f);
    rec[2 * j] = make_float4(x, y, z, (float)(a * u[n + j]));
    rec[2 * j + 1] = make_float4((float)(fphi * nx), (float)(fphi * ny), (float)(fphi * nz), 0.f);
  } else {
    rec[2 * j] = make_float4((float)kFarS, (float)kFarS, (float)kFarS, 0.f);
    rec[2 * j + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// grid = (tiles, splits): the same tiling as the handle-based FP32 mat-vec
__global__ void __launch_bounds__(kSNT) k_static_pairs(int n, int n_chunks, int chunks_per_split,
                                                       PairConst<float> c, unsigned char* __restrict__ scratch) {
  __shared__ float4 sh[2 * kSCH];
  const float4* tgt = reinterpret_cast<const float4*>(scratch + kOffTgt);
  const float4* rec = reinterpret_cast<const float4*>(scratch + kOffRec);
  float* part = reinterpret_cast<float*>(scratch + kOffPart);
  const int t0 = blockIdx.x * kSNT * kSTPT;
  float tx[kSTPT], ty[kSTPT], tz[kSTPT], nx[kSTPT], ny[kSTPT], nz[kSTPT], ap[kSTPT], aq[kSTPT];
  int idx[kSTPT];
#pragma unroll
  for (int k = 0; k < kSTPT; ++k) {
    idx[k] = t0 + k * kSNT + threadIdx.x;
    int i = min(idx[k], n - 1);
    float4 g = tgt[2 * i], v = tgt[2 * i + 1];
    tx[k] = g.x, ty[k] = g.y, tz[k] = g.z, nx[k] = v.x, ny[k] = v.y, nz[k] = v.z;
    ap[k] = 0.f, aq[k] = 0.f;
  }
  const int c0 = blockIdx.y * chunks_per_split, c1 = min(c0 + chunks_per_split, n_chunks);
  for (int ch = c0; ch < c1; ++ch) {
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * kSCH; q += kSNT) sh[q] = rec[(size_t)ch * 2 * kSCH + q];
    __syncthreads();
    const int j0 = ch * kSCH;
    const bool diag = (j0 < t0 + kSNT * kSTPT) && (j0 + kSCH > t0);
    for (int jj = 0; jj < kSCH; ++jj) {
      const float4 A = sh[2 * jj], B = sh[2 * jj + 1];
#pragma unroll
      for (int k = 0; k < kSTPT; ++k) {
        if (diag)
          pair_forward<true>(tx[k], ty[k], tz[k], nx[k], ny[k], nz[k], A.x, A.y, A.z, A.w, B.x, B.y, B.z,
                             j0 + jj == idx[k], c, ap[k], aq[k]);
        else
          pair_forward<false>(tx[k], ty[k], tz[k], nx[k], ny[k], nz[k], A.x, A.y, A.z, A.w, B.x, B.y, B.z,
                              false, c, ap[k], aq[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kSTPT; ++k)
    if (idx[k] < n) {
      part[(size_t)blockIdx.y * 2 * n + idx[k]] = ap[k];
      part[(size_t)blockIdx.y * 2 * n + n + idx[k]] = aq[k];
    }
}

__global__ void k_static_reduce(int n, int n_splits, const double* __restrict__ u, double* __restrict__ y,
                                double d_phi, double d_psi, const unsigned char* __restrict__ scratch) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  const float* part = reinterpret_cast<const float*>(scratch + kOffPart);
  double acc = 0.0;
  for (int sp = 0; sp < n_splits; ++sp) acc += (double)part[(size_t)sp * 2 * n + i];
  y[i] = (i < n ? d_phi : d_psi) * u[i] - kInv4PiS * acc;
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};
int g_static_sms[kMaxDevices] = {};

unsigned char* static_scratch(int dev, int* num_sms) {
  BIPB_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error(BIPB_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    BIPB_CUDA(cudaDeviceGetAttribute(&g_static_sms[dev], cudaDevAttrMultiProcessorCount, dev));
    g_static_addr[dev] = p;
  }
  *num_sms = g_static_sms[dev];
  return static_cast<unsigned char*>(g_static_addr[dev]);
}

}  // namespace
}  // namespace bipb

using namespace bipb;

extern "C" bipb_status bipb_matvec32_static(int64_t n, const double* centroids, const double* normals,
                                            const double* areas, const bipb_medium* m, const double* u,
                                            double* y, void* cuda_stream) {
  try {
    BIPB_REQUIRE(n >= 2, "need at least 2 triangles");
    if (n > kStaticMaxN)
      throw Error(BIPB_ERR_INVALID_ARG, "bipb_matvec32_static accepts at most 32768 triangles (its static "
                                        "scratch size); use a bipb_surface handle for larger surfaces");
    BIPB_REQUIRE(centroids && normals && areas && u && y, "NULL device pointer");
    BIPB_REQUIRE(u != y, "y must not alias u");
    BIPB_REQUIRE(m != nullptr, "medium is NULL");
    BIPB_REQUIRE(std::isfinite(m->eps_in) && m->eps_in > 0 && std::isfinite(m->eps_out) && m->eps_out > 0 &&
                     std::isfinite(m->kappa) && m->kappa >= 0,
                 "eps_in, eps_out must be > 0 and kappa >= 0");
    int dev = 0;
    BIPB_CUDA(cudaGetDevice(&dev));
    int num_sms = 0;
    unsigned char* scratch = static_scratch(dev, &num_sms);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int nn = (int)n;
    const int n_tiles = (nn + kSNT * kSTPT - 1) / (kSNT * kSTPT);
    const int n_chunks = (nn + kSCH - 1) / kSCH;
    int splits = std::max(1, (num_sms * 8 + n_tiles - 1) / n_tiles);
    splits = std::min({splits, std::max(1, n_chunks / 4), kStaticMaxSplits});
    const int cps = (n_chunks + splits - 1) / splits;
    splits = (n_chunks + cps - 1) / cps;
    const double eps = m->eps_out / m->eps_in;
    PairConst<float> c;
    c.eps = (float)eps;
    c.inveps = (float)(1.0 / eps);
    c.kappa = (float)m->kappa;
    c.nkl2e = (float)(-m->kappa * 1.4426950408889634);
    c.smax = kSMaxF;
    k_static_center<<<1, 256, 0, st>>>(nn, centroids, scratch);
    BIPB_CUDA(cudaGetLastError());
    const int n_pad = n_chunks * kSCH;
    k_static_pack<<<(n_pad + 255) / 256, 256, 0, st>>>(nn, n_pad, centroids, normals, areas, u, scratch);
    BIPB_CUDA(cudaGetLastError());
    k_static_pairs<<<dim3(n_tiles, splits), kSNT, 0, st>>>(nn, n_chunks, cps, c, scratch);
    BIPB_CUDA(cudaGetLastError());
    k_static_reduce<<<(2 * nn + 255) / 256, 256, 0, st>>>(nn, splits, u, y, 0.5 * (1.0 + eps),
                                                          0.5 * (1.0 + 1.0 / eps), scratch);
    BIPB_CUDA(cudaGetLastError());
    set_last_error("");
    return BIPB_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.st;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return BIPB_ERR_CUDA;
  }
}
