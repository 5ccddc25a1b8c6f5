// pic_static.cu -- Poisson solve on caller-provided device buffers that
// allocates nothing: its work vectors live in one file-scope device array.
//
// Some callers cannot call cudaMalloc while they run: a host program that
// hands out all device memory from its own pool up front, code running where
// allocation would synchronise the device or fragment a carefully sized heap,
// or a coupling driver that must not grow its footprint between steps. For them
// pic_poisson_solve_static solves the same discrete problem as pic_solve with
// conjugate gradients whose vectors (right-hand side, residual, search
// direction, operator image) and reduction partials sit in g_static_scratch.
//
// The array is a fixed PIC_STATIC_MAX_UNKNOWNS-sized allocation that every GPU
// loading this library holds until the process exits (4 vectors of 2^18
// doubles plus partials, 8.1 MiB). All calls share it and it keeps the last
// call's contents; every vector is written before it is read within a call, so
// nothing needs clearing between calls. Calls whose work overlaps on the GPU
// (different streams, or different host threads on one device) race on it.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace pic {

constexpr long long kStaticVec = PIC_STATIC_MAX_UNKNOWNS;
constexpr int kStaticBlock = 256;
constexpr int kStaticParts = 1024;  // block partials (grid size cap)
constexpr int kStaticScalars = 8;   // rr, pq, alpha, beta, bb

static __device__ __align__(256) double g_static_scratch[4 * kStaticVec + kStaticParts + kStaticScalars];

namespace {

struct StaticLv {
  int nx, ny, nz;
  long long pl, nu;
};

__device__ __forceinline__ double s_nb_sum(const StaticLv& L, const double* __restrict__ x, long long u) {
  const int k = (int)(u / L.pl);
  const long long r = u - (long long)k * L.pl;
  const int j = (int)(r / L.nx);
  const int i = (int)(r - (long long)j * L.nx);
  const long long row = u - i;
  const int im = i == 0 ? L.nx - 1 : i - 1, ip = i == L.nx - 1 ? 0 : i + 1;
  const long long rm = j == 0 ? (long long)(L.ny - 1) * L.nx : -(long long)L.nx;
  const long long rp = j == L.ny - 1 ? -(long long)(L.ny - 1) * L.nx : (long long)L.nx;
  double s = x[row + im] + x[row + ip] + x[u + rm] + x[u + rp];
  if (k > 0) s += x[u - L.pl];
  if (k < L.nz - 2) s += x[u + L.pl];
  return s;
}

__device__ __forceinline__ void s_block_partial(double v, double* part) {
  __shared__ double sm[kStaticBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kStaticBlock / 32; ++w) s += sm[w];
    part[blockIdx.x] = s;
  }
}

// b = h^2 rho / eps0 over the unknowns (+ electrode values on the planes next to them);
// phi's electrode planes are set; part = b.b
__global__ void k_static_rhs(StaticLv L, double h, double phi_c, double phi_a, const double* __restrict__ rho,
                             double* __restrict__ phi, double* __restrict__ b, double* part) {
  const double s = h * h / kEps0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < L.pl; p += (long long)gridDim.x * blockDim.x) {
    phi[p] = phi_c;
    phi[(long long)L.nz * L.pl + p] = phi_a;
  }
  double acc = 0.0;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < L.nu; u += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(u / L.pl) + 1;
    double v = s * rho[u + L.pl];
    if (k == 1) v += phi_c;
    if (k == L.nz - 1) v += phi_a;
    b[u] = v;
    acc += v * v;
  }
  s_block_partial(acc, part);
}

// r = b - A x ; p = r ; part = r.r
__global__ void k_static_residual(StaticLv L, const double* __restrict__ x, const double* __restrict__ b,
                                  double* __restrict__ r, double* __restrict__ p, double* part) {
  double acc = 0.0;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < L.nu; u += (long long)gridDim.x * blockDim.x) {
    const double v = b[u] - (6.0 * x[u] - s_nb_sum(L, x, u));
    r[u] = v;
    p[u] = v;
    acc += v * v;
  }
  s_block_partial(acc, part);
}

// q = A p ; part = p.q
__global__ void k_static_apply(StaticLv L, const double* __restrict__ p, double* __restrict__ q, double* part) {
  double acc = 0.0;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < L.nu; u += (long long)gridDim.x * blockDim.x) {
    const double v = 6.0 * p[u] - s_nb_sum(L, p, u);
    q[u] = v;
    acc += p[u] * v;
  }
  s_block_partial(acc, part);
}

// x += alpha p ; r -= alpha q ; part = r.r
__global__ void k_static_update(StaticLv L, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                                const double* __restrict__ q, const double* sc, double* part) {
  const double alpha = sc[2];
  double acc = 0.0;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < L.nu; u += (long long)gridDim.x * blockDim.x) {
    x[u] += alpha * p[u];
    const double v = r[u] - alpha * q[u];
    r[u] = v;
    acc += v * v;
  }
  s_block_partial(acc, part);
}

// p = r + beta p
__global__ void k_static_direction(StaticLv L, double* __restrict__ p, const double* __restrict__ r, const double* sc) {
  const double beta = sc[3];
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < L.nu; u += (long long)gridDim.x * blockDim.x)
    p[u] = r[u] + beta * p[u];
}

// scalar bookkeeping in a fixed order: which = 0 (bb), 1 (initial rr), 2 (pq -> alpha), 3 (new rr -> beta)
__global__ void k_static_scalars(const double* part, int nparts, double* sc, int which) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < nparts; ++i) s += part[i];
  if (which == 0) {
    sc[4] = s;
  } else if (which == 1) {
    sc[0] = s;
  } else if (which == 2) {
    sc[1] = s;
    sc[2] = s != 0.0 ? sc[0] / s : 0.0;
  } else {
    sc[3] = sc[0] != 0.0 ? s / sc[0] : 0.0;
    sc[0] = s;
  }
}

std::mutex g_setup_mutex;
double* g_scratch_ptr[64] = {nullptr};

// Device address of g_static_scratch for the current device (set-up on first use).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace pic

using namespace pic;

namespace pic {
void set_static_error(const char* msg);  // pic_api.cu: text for pic_last_error(NULL)
}

extern "C" pic_status pic_poisson_solve_static(int32_t nx, int32_t ny, int32_t nz, double h, double phi_cathode_V,
                                               double phi_anode_V, const double* rho_dev, double* phi_dev, double rtol,
                                               int32_t maxit, void* cuda_stream, int32_t* iters, double* resid_rel) {
  if (nx < 1 || ny < 1 || nz < 2 || !(h > 0) || !(rtol > 0) || maxit < 1 || !rho_dev || !phi_dev) {
    set_static_error("pic_poisson_solve_static: need nx, ny >= 1, nz >= 2, h > 0, rtol > 0, maxit >= 1 and both arrays");
    return PIC_EINVAL;
  }
  const long long nu = (long long)nx * ny * (nz - 1);
  if (nu > kStaticVec) {
    set_static_error("pic_poisson_solve_static: nx*ny*(nz-1) exceeds PIC_STATIC_MAX_UNKNOWNS (262144)");
    return PIC_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) {
    set_static_error("pic_poisson_solve_static: cudaGetSymbolAddress of the fixed work array failed");
    return PIC_ECUDA;
  }
  double* b = base;
  double* r = base + kStaticVec;
  double* p = base + 2 * kStaticVec;
  double* q = base + 3 * kStaticVec;
  double* part = base + 4 * kStaticVec;
  double* sc = part + kStaticParts;
  const StaticLv L{nx, ny, nz, (long long)nx * ny, nu};
  long long gb = (nu + kStaticBlock - 1) / kStaticBlock;
  const int G = (int)(gb < 1 ? 1 : (gb > kStaticParts ? kStaticParts : gb));
  double* x = phi_dev + L.pl;  // unknown nodes k = 1..nz-1 are contiguous

  // A failed launch leaves no sticky error and the scalars keep the previous
  // call's values, so every read of a decision scalar is preceded by a check of
  // the launches before it.
  auto fail = [&](const char* what, cudaError_t e) -> pic_status {
    char msg[256];
    snprintf(msg, sizeof msg, "pic_poisson_solve_static: %s: %s", what, cudaGetErrorString(e));
    set_static_error(msg);
    return PIC_ECUDA;
  };
  auto read = [&](int idx, double* out) -> cudaError_t {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(out, sc + idx, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
  };
  // a launch error left by earlier, unrelated work is cleared, not reported as this call's
  cudaError_t e = cudaGetLastError();
  PIC_LAUNCH(G, kStaticBlock, 0, s, k_static_rhs)(L, h, phi_cathode_V, phi_anode_V, rho_dev, phi_dev, b, part);
  PIC_LAUNCH(1, 1, 0, s, k_static_scalars)(part, G, sc, 0);
  PIC_LAUNCH(G, kStaticBlock, 0, s, k_static_residual)(L, x, b, r, p, part);
  PIC_LAUNCH(1, 1, 0, s, k_static_scalars)(part, G, sc, 1);
  double bb = 0.0, rr = 0.0;
  if ((e = read(4, &bb)) != cudaSuccess) return fail("right-hand side", e);
  if ((e = read(0, &rr)) != cudaSuccess) return fail("initial residual", e);
  const double tol = rtol * std::sqrt(bb);
  int it = 0;
  if (bb > 0.0) {
    while (std::sqrt(rr) > tol && it < maxit) {
      PIC_LAUNCH(G, kStaticBlock, 0, s, k_static_apply)(L, p, q, part);
      PIC_LAUNCH(1, 1, 0, s, k_static_scalars)(part, G, sc, 2);
      PIC_LAUNCH(G, kStaticBlock, 0, s, k_static_update)(L, x, r, p, q, sc, part);
      PIC_LAUNCH(1, 1, 0, s, k_static_scalars)(part, G, sc, 3);
      PIC_LAUNCH(G, kStaticBlock, 0, s, k_static_direction)(L, p, r, sc);
      ++it;
      if ((e = read(0, &rr)) != cudaSuccess) return fail("CG iteration", e);
      if (!std::isfinite(rr)) break;
    }
    // the status follows the true residual b - A x, recomputed here
    PIC_LAUNCH(G, kStaticBlock, 0, s, k_static_residual)(L, x, b, r, p, part);
    PIC_LAUNCH(1, 1, 0, s, k_static_scalars)(part, G, sc, 1);
    if ((e = read(0, &rr)) != cudaSuccess) return fail("true residual", e);
  } else {
    if ((e = cudaMemsetAsync(x, 0, sizeof(double) * nu, s)) != cudaSuccess) return fail("zero solution", e);
    rr = 0.0;
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail("stream synchronise", e);
  const double rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  if (iters) *iters = it;
  if (resid_rel) *resid_rel = rel;
  if (!(rel <= rtol)) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "pic_poisson_solve_static: true relative residual %.3e above rtol %.3e after %d iterations", rel, rtol,
             it);
    set_static_error(msg);
    return PIC_ENOCONV;
  }
  return PIC_OK;
}
