// k_solver.cu -- Poisson solve of Eq. (1) on the node grid (a4).
//
// Unknowns: nodes k = 1..nz-1 (periodic i, j); operator scaled by h^2:
//   (A x)_ijk = 6 x_ijk - sum of the six neighbours (Dirichlet planes folded into b).
// Solver: conjugate gradients preconditioned by one geometric-multigrid V(1,1)
// cycle: red-black Gauss-Seidel (pre-smoothing red then black, post-smoothing
// black then red, so the cycle is a symmetric operator), full-weighting
// restriction (b_coarse = 4 FW(r_fine) for the h^2 scaling), trilinear
// prolongation, coarsest level solved exactly with a dense inverse.
//  - FP64 path: everything in FP64.
//  - MIXED path: iterative refinement; the residual r = b - A x and the update
//    x += d are FP64, the correction d solves A d = r with the same PCG in FP32
//    (FP32 smoothing and transfer operators), to a loose inner tolerance.
// Dot products are reduced per block then summed in a fixed order on the
// device; the host reads one residual norm per iteration to stop.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "pic_internal.cuh"
#include "pic_kernels.cuh"
#include "pic_solver.cuh"

namespace pic {

constexpr int kSB = 256;
constexpr int kMaxRedBlocks = 152 * 8;

static int sgrid(long long n) {
  long long b = (n + kSB - 1) / kSB;
  if (b < 1) b = 1;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
  return (int)b;
}

struct Lv {
  int nx, ny, nz;
  long long pl, nu;
};
static Lv lv_of(const MgLevel& L) { return Lv{L.nx, L.ny, L.nz, (long long)L.nx * L.ny, L.nu}; }

template <class T>
__device__ __forceinline__ T nb_sum(const Lv& L, const T* __restrict__ x, long long u, int i, int j, int k) {
  // k: unknown plane index 0..nz-2
  const long long row = u - i;
  const int im = i == 0 ? L.nx - 1 : i - 1, ip = i == L.nx - 1 ? 0 : i + 1;
  const long long rm = (j == 0 ? (long long)(L.ny - 1) * L.nx : -(long long)L.nx);
  const long long rp = (j == L.ny - 1 ? -(long long)(L.ny - 1) * L.nx : (long long)L.nx);
  T s = x[row + im] + x[row + ip] + x[u + rm] + x[u + rp];
  if (k > 0) s += x[u - L.pl];
  if (k < L.nz - 2) s += x[u + L.pl];
  return s;
}

__device__ __forceinline__ void uijk(const Lv& L, long long u, int& i, int& j, int& k) {
  k = (int)(u / L.pl);
  const long long r = u - (long long)k * L.pl;
  j = (int)(r / L.nx);
  i = (int)(r - (long long)j * L.nx);
}

template <class T, class Acc>
__device__ __forceinline__ void block_partial(Acc v, double* part) {
  __shared__ double sm[kSB / 32];
  double d = (double)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kSB / 32; ++w) s += sm[w];
    part[blockIdx.x] = s;
  }
}

// y = A x ; part = x . y
template <class T>
__global__ void __launch_bounds__(kSB) k_apply_dot(Lv L, const T* __restrict__ x, T* __restrict__ y, double* part) {
  T acc = 0;
  for (long long u = gtid(); u < L.nu; u += gstride()) {
    int i, j, k;
    uijk(L, u, i, j, k);
    const T xv = x[u];
    const T yv = (T)6 * xv - nb_sum(L, x, u, i, j, k);
    y[u] = yv;
    acc += xv * yv;
  }
  block_partial<T, T>(acc, part);
}

// r = b - A x ; part = r . r  (Tx/Tb may be FP64 while r is FP32 for the mixed residual)
template <class Tx, class Tr>
__global__ void __launch_bounds__(kSB) k_residual(Lv L, const Tx* __restrict__ x, const Tx* __restrict__ b,
                                                  Tr* __restrict__ r, double* part) {
  Tx acc = 0;
  for (long long u = gtid(); u < L.nu; u += gstride()) {
    int i, j, k;
    uijk(L, u, i, j, k);
    const Tx rv = b[u] - ((Tx)6 * x[u] - nb_sum(L, x, u, i, j, k));
    r[u] = (Tr)rv;
    acc += rv * rv;
  }
  if (part) block_partial<Tx, Tx>(acc, part);
}

// partial dot a . b
template <class T>
__global__ void __launch_bounds__(kSB) k_dot(long long n, const T* __restrict__ a, const T* __restrict__ b, double* part) {
  T acc = 0;
  for (long long u = gtid(); u < n; u += gstride()) acc += a[u] * b[u];
  block_partial<T, T>(acc, part);
}

// ---------------------------------------------------------------------------
// multigrid pieces
// ---------------------------------------------------------------------------
// One red-black Gauss-Seidel half sweep: points with (i + j + knode) % 2 == color.
// zero_init: the level starts from e = 0 (the other colour is written as 0).
template <class T>
__global__ void __launch_bounds__(kSB) k_smooth(Lv L, T* __restrict__ e, const T* __restrict__ b, int color, int zero_init) {
  const int hx = L.nx >> 1;
  const long long npts = L.nu >> 1;
  const T sixth = (T)(1.0 / 6.0);
  for (long long t = gtid(); t < npts; t += gstride()) {
    const long long row = t / hx;
    const int m = (int)(t - row * hx);
    const int j = (int)(row % L.ny);
    const int k = (int)(row / L.ny);  // unknown plane (node k+1)
    const int par = (j + k + 1 + color) & 1;
    const int i = 2 * m + par;
    const long long u = (long long)k * L.pl + (long long)j * L.nx + i;
    if (zero_init) {
      e[u] = b[u] * sixth;
      e[u - i + (2 * m + (par ^ 1))] = (T)0;
    } else {
      e[u] = (b[u] + nb_sum(L, e, u, i, j, k)) * sixth;
    }
  }
}

// b_c = 4 * full-weighting(r_f) on coarse unknowns
template <class T>
__global__ void __launch_bounds__(kSB) k_restrict(Lv F, Lv Cc, const T* __restrict__ r, T* __restrict__ bc) {
  for (long long u = gtid(); u < Cc.nu; u += gstride()) {
    int I, J, K;
    uijk(Cc, u, I, J, K);
    const int Kn = K + 1;  // coarse node index
    T s = 0;
#pragma unroll
    for (int c = -1; c <= 1; ++c) {
      const int kf = 2 * Kn + c - 1;  // fine unknown plane
      const T wc = c == 0 ? (T)0.5 : (T)0.25;
#pragma unroll
      for (int b2 = -1; b2 <= 1; ++b2) {
        int jf = 2 * J + b2;
        jf = jf < 0 ? jf + F.ny : (jf >= F.ny ? jf - F.ny : jf);
        const T wb = b2 == 0 ? (T)0.5 : (T)0.25;
        const long long rowf = (long long)kf * F.pl + (long long)jf * F.nx;
#pragma unroll
        for (int a2 = -1; a2 <= 1; ++a2) {
          int iff = 2 * I + a2;
          iff = iff < 0 ? iff + F.nx : (iff >= F.nx ? iff - F.nx : iff);
          const T wa = a2 == 0 ? (T)0.5 : (T)0.25;
          s += wa * wb * wc * r[rowf + iff];
        }
      }
    }
    bc[u] = (T)4 * s;
  }
}

// e_f += P e_c (trilinear; coarse Dirichlet planes carry 0)
template <class T>
__global__ void __launch_bounds__(kSB) k_prolong(Lv F, Lv Cc, const T* __restrict__ ec, T* __restrict__ ef) {
  for (long long u = gtid(); u < F.nu; u += gstride()) {
    int i, j, k;
    uijk(F, u, i, j, k);
    const int kn = k + 1;  // fine node
    const int I0 = i >> 1, J0 = j >> 1, K0 = kn >> 1;
    const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (kn & 1) ? 2 : 1;
    const T w = (T)1 / (T)(ni * nj * nk);
    T s = 0;
    const int I1 = I0 + 1 == Cc.nx ? 0 : I0 + 1;
    const int J1 = J0 + 1 == Cc.ny ? 0 : J0 + 1;
    for (int c = 0; c < nk; ++c) {
      const int K = K0 + c;  // coarse node
      if (K <= 0 || K >= Cc.nz) continue;
      const long long pk = (long long)(K - 1) * Cc.pl;
      for (int b2 = 0; b2 < nj; ++b2) {
        const long long row = pk + (long long)(b2 ? J1 : J0) * Cc.nx;
        s += ec[row + I0];
        if (ni == 2) s += ec[row + I1];
      }
    }
    ef[u] += w * s;
  }
}

// coarsest level: e = Ainv b (dense, row per warp)
template <class T>
__global__ void k_coarse(long long n, const T* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ e) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < n; r += nwarps) {
    T s = 0;
    for (long long c = lane; c < n; c += 32) s += Ainv[r * n + c] * b[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) e[r] = s;
  }
}

template <class T>
__global__ void k_axpy_cast(long long n, double* __restrict__ x, const T* __restrict__ d) {
  for (long long u = gtid(); u < n; u += gstride()) x[u] += (double)d[u];
}
template <class T>
__global__ void k_zero(long long n, T* __restrict__ x) {
  for (long long u = gtid(); u < n; u += gstride()) x[u] = (T)0;
}
template <class T>
__global__ void k_copy(long long n, T* __restrict__ d, const T* __restrict__ s) {
  for (long long u = gtid(); u < n; u += gstride()) d[u] = s[u];
}

__global__ void k_copy_cast(long long n, float* __restrict__ d, const double* __restrict__ s) {
  for (long long u = gtid(); u < n; u += gstride()) d[u] = (float)s[u];
}
template <class T>
__global__ void k_jacobi_scale(long long n, T* z) {
  for (long long u = gtid(); u < n; u += gstride()) z[u] *= (T)(1.0 / 6.0);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static std::vector<double> dense_inverse(const MgLevel& L) {
  const long long n = L.nu;
  std::vector<double> A((size_t)(n * n), 0.0), I((size_t)(n * n), 0.0);
  const long long pl = (long long)L.nx * L.ny;
  for (long long u = 0; u < n; ++u) {
    const int k = (int)(u / pl);
    const long long r = u - k * pl;
    const int j = (int)(r / L.nx), i = (int)(r - (long long)j * L.nx);
    A[u * n + u] += 6.0;
    const int im = (i + L.nx - 1) % L.nx, ip = (i + 1) % L.nx;
    const int jm = (j + L.ny - 1) % L.ny, jp = (j + 1) % L.ny;
    A[u * n + (k * pl + (long long)j * L.nx + im)] -= 1.0;
    A[u * n + (k * pl + (long long)j * L.nx + ip)] -= 1.0;
    A[u * n + (k * pl + (long long)jm * L.nx + i)] -= 1.0;
    A[u * n + (k * pl + (long long)jp * L.nx + i)] -= 1.0;
    if (k > 0) A[u * n + (u - pl)] -= 1.0;
    if (k < L.nz - 2) A[u * n + (u + pl)] -= 1.0;
    I[u * n + u] = 1.0;
  }
  // Gauss-Jordan with partial pivoting (SPD, small)
  for (long long c = 0; c < n; ++c) {
    long long p = c;
    for (long long r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    if (p != c)
      for (long long q = 0; q < n; ++q) {
        std::swap(A[c * n + q], A[p * n + q]);
        std::swap(I[c * n + q], I[p * n + q]);
      }
    const double d = 1.0 / A[c * n + c];
    for (long long q = 0; q < n; ++q) {
      A[c * n + q] *= d;
      I[c * n + q] *= d;
    }
    for (long long r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      if (f == 0.0) continue;
      for (long long q = 0; q < n; ++q) {
        A[r * n + q] -= f * A[c * n + q];
        I[r * n + q] -= f * I[c * n + q];
      }
    }
  }
  // symmetrise against rounding
  for (long long r = 0; r < n; ++r)
    for (long long c = r + 1; c < n; ++c) {
      const double m = 0.5 * (I[r * n + c] + I[c * n + r]);
      I[r * n + c] = I[c * n + r] = m;
    }
  return I;
}

std::vector<MgLevel> mg_plan(int nx, int ny, int nz) {
  std::vector<MgLevel> lv;
  MgLevel L{nx, ny, nz, (long long)nx * ny * (nz - 1)};
  lv.push_back(L);
  const bool rb_ok = (nx % 2 == 0) && (ny % 2 == 0);
  if (!rb_ok) return lv;
  while (true) {
    const MgLevel& c = lv.back();
    if (c.nu <= 512) break;
    if (c.nx % 2 || c.ny % 2 || c.nz % 2) break;
    if (c.nx < 8 || c.ny < 8 || c.nz < 8) break;
    MgLevel n{c.nx / 2, c.ny / 2, c.nz / 2, (long long)(c.nx / 2) * (c.ny / 2) * (c.nz / 2 - 1)};
    if ((n.nx % 2) || (n.ny % 2)) break;
    lv.push_back(n);
  }
  return lv;
}

template <class T>
cudaError_t Mg<T>::init(const std::vector<MgLevel>& plan) {
  levels = plan;
  rb_ok = (plan[0].nx % 2 == 0) && (plan[0].ny % 2 == 0);
  const size_t nl = plan.size();
  e.assign(nl, nullptr);
  b.assign(nl, nullptr);
  r.assign(nl, nullptr);
  cudaError_t err = cudaSuccess;
  for (size_t l = 0; l < nl; ++l) {
    const size_t bytes = sizeof(T) * (size_t)(plan[l].nu > 0 ? plan[l].nu : 1);
    if (l > 0) {
      if ((err = cudaMalloc(&e[l], bytes))) return err;
      if ((err = cudaMalloc(&b[l], bytes))) return err;
    }
    if ((err = cudaMalloc(&r[l], bytes))) return err;
  }
  const MgLevel& c = plan.back();
  coarse_dense = rb_ok && c.nu <= 1024 && nl >= 1;
  if (coarse_dense) {
    std::vector<double> inv = dense_inverse(c);
    std::vector<T> invT(inv.begin(), inv.end());
    if ((err = cudaMalloc(&Ainv, sizeof(T) * invT.size()))) return err;
    if ((err = cudaMemcpy(Ainv, invT.data(), sizeof(T) * invT.size(), cudaMemcpyHostToDevice))) return err;
  }
  return cudaSuccess;
}

template <class T>
void Mg<T>::release() {
  for (auto* p : e) cudaFree(p);
  for (auto* p : b) cudaFree(p);
  for (auto* p : r) cudaFree(p);
  e.clear();
  b.clear();
  r.clear();
  if (Ainv) cudaFree(Ainv);
  Ainv = nullptr;
}

// z = M^-1 rhs (one V(1,1) cycle from zero); rhs and z live at level 0 outside
template <class T>
void Mg<T>::vcycle(const T* rhs, T* z, cudaStream_t s) {
  const int nl = (int)levels.size();
  if (!rb_ok) {
    // Jacobi preconditioner: z = rhs / 6
    const Lv L = lv_of(levels[0]);
    PIC_LAUNCH(sgrid(L.nu), kSB, 0, s, k_copy<T>)(L.nu, z, rhs);
    PIC_LAUNCH(sgrid(L.nu), kSB, 0, s, k_jacobi_scale<T>)(L.nu, z);
    return;
  }
  std::vector<T*> E(nl), B(nl);
  for (int l = 0; l < nl; ++l) {
    E[l] = l == 0 ? z : e[l];
    B[l] = l == 0 ? const_cast<T*>(rhs) : b[l];
  }
  for (int l = 0; l < nl - 1; ++l) {
    const Lv L = lv_of(levels[l]);
    const long long half = L.nu >> 1;
    PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(L, E[l], B[l], 0, 1);
    PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(L, E[l], B[l], 1, 0);
    PIC_LAUNCH(sgrid(L.nu), kSB, 0, s, k_residual<T, T>)(L, E[l], B[l], r[l], nullptr);
    const Lv C = lv_of(levels[l + 1]);
    PIC_LAUNCH(sgrid(C.nu), kSB, 0, s, k_restrict<T>)(L, C, r[l], B[l + 1]);
  }
  {
    const Lv C = lv_of(levels[nl - 1]);
    if (coarse_dense) {
      const int cg = (int)std::min<long long>((C.nu * 32 + kSB - 1) / kSB, 4096);
      PIC_LAUNCH(cg, kSB, 0, s, k_coarse<T>)(C.nu, Ainv, B[nl - 1],
                                                                                              E[nl - 1]);
    } else {
      const long long half = C.nu >> 1;
      PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 0, 1);
      PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 1, 0);
      for (int it = 0; it < coarse_sweeps; ++it) {
        PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 1, 0);
        PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 0, 0);
        PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 0, 0);
        PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 1, 0);
      }
      PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 1, 0);
      PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 0, 0);
    }
  }
  for (int l = nl - 2; l >= 0; --l) {
    const Lv L = lv_of(levels[l]);
    const Lv C = lv_of(levels[l + 1]);
    PIC_LAUNCH(sgrid(L.nu), kSB, 0, s, k_prolong<T>)(L, C, E[l + 1], E[l]);
    const long long half = L.nu >> 1;
    PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(L, E[l], B[l], 1, 0);
    PIC_LAUNCH(sgrid(half), kSB, 0, s, k_smooth<T>)(L, E[l], B[l], 0, 0);
  }
}

// ---------------------------------------------------------------------------
// Device-controlled solve. All scalars live in SolveCtl on the device; the
// stopping decisions set the conditional handles of two nested WHILE nodes of a
// CUDA graph (outer: FP64 true residual / refinement; inner: PCG iterations),
// so a solve is one graph launch with no host round trip.
// ---------------------------------------------------------------------------
constexpr int kFinBlock = 512;
// Sum of the block partials by one block of kFinBlock threads, in a fixed order
// (strided per-thread sums, then a shared-memory tree); returns the total in
// every thread.
__device__ __forceinline__ double sum_parts(const double* part, int n) {
  __shared__ double sm[kFinBlock];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kFinBlock) s += part[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = kFinBlock / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  const double t = sm[0];
  __syncthreads();
  return t;
}

__global__ void k_fin_bb(const double* part, int nparts, SolveCtl* c, double rtol, int maxit) {
  const double bb = sum_parts(part, nparts);
  if (threadIdx.x != 0) return;
  c->bb = bb;
  c->tol2 = rtol * rtol * bb;
  c->it_total = 0;
  c->outer = 0;
  c->converged = bb == 0.0 ? 1 : 0;
  c->maxit = maxit;
  c->rr_true = 0.0;
  c->resid_rel = 0.0;
}

// r_in = (Tin)(b - A x) with x, b FP64; d = 0; partial sums of r.r (FP64)
template <class Tin>
__global__ void __launch_bounds__(kSB) k_residual_prep(Lv L, const double* __restrict__ x, const double* __restrict__ b,
                                                       Tin* __restrict__ r_in, Tin* __restrict__ d, double* part,
                                                       const SolveCtl* c) {
  double acc = 0.0;
  const bool zero_x = c->bb == 0.0;
  for (long long u = gtid(); u < L.nu; u += gstride()) {
    int i, j, k;
    uijk(L, u, i, j, k);
    const double rv = zero_x ? 0.0 : b[u] - (6.0 * x[u] - nb_sum(L, x, u, i, j, k));
    r_in[u] = (Tin)rv;
    d[u] = (Tin)0;
    acc += rv * rv;
  }
  block_partial<double, double>(acc, part);
}

__global__ void k_fin_outer(const double* part, int nparts, SolveCtl* c, cudaGraphConditionalHandle h_outer,
                            cudaGraphConditionalHandle h_inner, double inner_rtol, int mixed, int max_outer, int use_graph) {
  const double rr = sum_parts(part, nparts);
  if (threadIdx.x != 0) return;
  c->rr_true = rr;
  c->resid_rel = c->bb > 0.0 ? sqrt(rr / c->bb) : 0.0;
  const bool done = c->bb == 0.0 || rr <= c->tol2 || !(rr == rr) || c->it_total >= c->maxit || c->outer >= max_outer;
  c->converged = (c->bb == 0.0 || rr <= c->tol2) ? 1 : 0;
  c->rr = rr;
  c->it_inner = 0;
  c->tol_in2 = mixed ? fmax(inner_rtol * inner_rtol * rr, 0.25 * c->tol2) : c->tol2;
  c->outer += 1;
  c->more = done ? 0 : 1;
  if (use_graph) {
    cudaGraphSetConditional(h_outer, done ? 0u : 1u);
    cudaGraphSetConditional(h_inner, done ? 0u : 1u);
  }
}

__global__ void k_fin_rz(const double* part, int nparts, SolveCtl* c) {
  const double rz = sum_parts(part, nparts);
  if (threadIdx.x != 0) return;
  c->beta = c->it_inner > 0 ? rz / c->rz : 0.0;
  c->rz = rz;
}

__global__ void k_fin_pq(const double* part, int nparts, SolveCtl* c) {
  const double pq = sum_parts(part, nparts);
  if (threadIdx.x != 0) return;
  c->pq = pq;
  c->alpha = pq != 0.0 ? c->rz / pq : 0.0;
}

__global__ void k_fin_rr(const double* part, int nparts, SolveCtl* c, cudaGraphConditionalHandle h_inner, int use_graph) {
  const double rr = sum_parts(part, nparts);
  if (threadIdx.x != 0) return;
  c->rr = rr;
  c->it_inner += 1;
  c->it_total += 1;
  const bool more = rr > c->tol_in2 && c->it_total < c->maxit && (rr == rr);
  c->more = more ? 1 : 0;
  if (use_graph) cudaGraphSetConditional(h_inner, more ? 1u : 0u);
}

// p = z (first iteration of this inner solve) or z + beta p
template <class T>
__global__ void __launch_bounds__(kSB) k_pupdate_c(long long n, T* __restrict__ p, const T* __restrict__ z, const SolveCtl* c) {
  const bool first = c->it_inner == 0;
  const T beta = (T)c->beta;
  for (long long u = gtid(); u < n; u += gstride()) p[u] = first ? z[u] : z[u] + beta * p[u];
}

// d += alpha p ; r -= alpha q ; partial r.r
template <class T>
__global__ void __launch_bounds__(kSB) k_update_c(long long n, T* __restrict__ d, T* __restrict__ r, const T* __restrict__ p,
                                                  const T* __restrict__ q, const SolveCtl* c, double* part) {
  const T alpha = (T)c->alpha;
  T acc = 0;
  for (long long u = gtid(); u < n; u += gstride()) {
    d[u] += alpha * p[u];
    const T rv = r[u] - alpha * q[u];
    r[u] = rv;
    acc += rv * rv;
  }
  block_partial<T, T>(acc, part);
}

// x += d (FP64); optionally phi32 = (float)(x - phi_vac(z)) on the same nodes
template <class T>
__global__ void __launch_bounds__(kSB) k_axpy_out(Lv L, double* __restrict__ x, const T* __restrict__ d, float* __restrict__ phi32,
                                                  double phi_c, double dphi_dk) {
  for (long long u = gtid(); u < L.nu; u += gstride()) {
    const double v = x[u] + (double)d[u];
    x[u] = v;
    if (phi32) {
      const int k = (int)(u / L.pl) + 1;  // node plane
      phi32[u] = (float)(v - (phi_c + dphi_dk * (double)k));
    }
  }
}

// ---------------------------------------------------------------------------
// host side: buffers
// ---------------------------------------------------------------------------
template <class T>
cudaError_t Pcg<T>::init(const std::vector<MgLevel>& plan) {
  n = plan[0].nu;
  cudaError_t err;
  const size_t bytes = sizeof(T) * (size_t)(n > 0 ? n : 1);
  if ((err = cudaMalloc(&r, bytes))) return err;
  if ((err = cudaMalloc(&z, bytes))) return err;
  if ((err = cudaMalloc(&p, bytes))) return err;
  if ((err = cudaMalloc(&q, bytes))) return err;
  if ((err = cudaMalloc(&d, bytes))) return err;
  if ((err = cudaMemset(p, 0, bytes))) return err;
  if ((err = cudaMemset(d, 0, bytes))) return err;
  return mg.init(plan);
}

template <class T>
void Pcg<T>::release() {
  cudaFree(r);
  cudaFree(z);
  cudaFree(p);
  cudaFree(q);
  cudaFree(d);
  r = z = p = q = d = nullptr;
  mg.release();
}

template struct Mg<double>;
template struct Mg<float>;
template struct Pcg<double>;
template struct Pcg<float>;

cudaError_t Solver::init(int nx, int ny, int nz, int precision_) {
  precision = precision_;
  plan = mg_plan(nx, ny, nz);
  n = plan[0].nu;
  cudaError_t err;
  if ((err = cudaMalloc(&b, sizeof(double) * (size_t)(n > 0 ? n : 1)))) return err;
  if ((err = cudaMemset(b, 0, sizeof(double) * (size_t)(n > 0 ? n : 1)))) return err;
  if ((err = cudaMalloc(&part, sizeof(double) * kMaxRedBlocks))) return err;
  if ((err = cudaMalloc(&ctl, sizeof(SolveCtl)))) return err;
  if ((err = cudaMemset(ctl, 0, sizeof(SolveCtl)))) return err;
  if ((err = cudaMallocHost(&host_ctl, sizeof(SolveCtl)))) return err;
  memset(host_ctl, 0, sizeof(SolveCtl));
  if (precision == 0) return p64.init(plan);
  return p32.init(plan);
}

void Solver::release() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  cudaFree(b);
  cudaFree(part);
  cudaFree(ctl);
  if (host_ctl) cudaFreeHost(host_ctl);
  host_ctl = nullptr;
  b = nullptr;
  part = nullptr;
  ctl = nullptr;
  p64.release();
  p32.release();
}

// One PCG iteration on the level-0 vectors of `pc` (captured into the inner body).
template <class T>
static void capture_pcg_iteration(Pcg<T>& pc, const Lv& L, double* part, SolveCtl* ctl,
                                  cudaGraphConditionalHandle h_inner, cudaStream_t s, int use_graph = 1) {
  const int G = sgrid(L.nu);
  pc.mg.vcycle(pc.r, pc.z, s);
  PIC_LAUNCH(G, kSB, 0, s, k_dot<T>)(L.nu, pc.r, pc.z, part);
  PIC_LAUNCH(1, kFinBlock, 0, s, k_fin_rz)(part, G, ctl);
  PIC_LAUNCH(G, kSB, 0, s, k_pupdate_c<T>)(L.nu, pc.p, pc.z, ctl);
  PIC_LAUNCH(G, kSB, 0, s, k_apply_dot<T>)(L, pc.p, pc.q, part);
  PIC_LAUNCH(1, kFinBlock, 0, s, k_fin_pq)(part, G, ctl);
  PIC_LAUNCH(G, kSB, 0, s, k_update_c<T>)(L.nu, pc.d, pc.r, pc.p, pc.q, ctl, part);
  PIC_LAUNCH(1, kFinBlock, 0, s, k_fin_rr)(part, G, ctl, h_inner, use_graph);
}

// Add a WHILE node at the current capture position of `s`; returns its body graph.
static cudaError_t add_while(cudaStream_t s, cudaGraphConditionalHandle* h, unsigned default_value, cudaGraph_t* body) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &status, nullptr, &g, &deps, &edges, &ndeps);
  if (e != cudaSuccess) return e;
  if (status != cudaStreamCaptureStatusActive) return cudaErrorIllegalState;
  e = cudaGraphConditionalHandleCreate(h, g, default_value, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = *h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, edges, ndeps, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Record the solve of A x = b (x = unknown view of phi) for this instance.
cudaError_t Solver::build_graph(double* x, float* phi32, double phi_c, double phi_a, int nz, double rtol, int maxit) {
  if (exec) return cudaSuccess;
  hx = x;
  hphi32 = phi32;
  h_phi_c = phi_c;
  h_dphi_dk = (phi_a - phi_c) / (double)nz;
  h_rtol = rtol;
  h_maxit = maxit;
  const char* env = getenv("PIC_SOLVER_GRAPH");
  if (env && env[0] == '0') return cudaSuccess;  // host-driven loop (profilers cannot see conditional graphs)
  const Lv L = lv_of(plan[0]);
  const int G = sgrid(L.nu);
  const int mixed = precision != 0;
  const double dphi_dk = (phi_a - phi_c) / (double)nz;
  cudaStream_t s0 = nullptr, s1 = nullptr, s2 = nullptr;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking))) return e;
  if ((e = cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking))) return e;
  if ((e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking))) return e;
  cudaGraphConditionalHandle h_outer, h_inner;
  cudaGraph_t outer_body = nullptr, inner_body = nullptr;
  e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    PIC_LAUNCH(G, kSB, 0, s0, k_dot<double>)(L.nu, b, b, part);
    PIC_LAUNCH(1, kFinBlock, 0, s0, k_fin_bb)(part, G, ctl, rtol, maxit);
    e = add_while(s0, &h_outer, 1u, &outer_body);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s1, outer_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      if (mixed) {
        PIC_LAUNCH(G, kSB, 0, s1, k_residual_prep<float>)(L, x, b, p32.r, p32.d, part, ctl);
      } else {
        PIC_LAUNCH(G, kSB, 0, s1, k_residual_prep<double>)(L, x, b, p64.r, p64.d, part, ctl);
      }
      e = cudaGraphConditionalHandleCreate(&h_inner, outer_body, 0u, 0);
      if (e == cudaSuccess)
        PIC_LAUNCH(1, kFinBlock, 0, s1, k_fin_outer)(part, G, ctl, h_outer, h_inner, inner_rtol, mixed, max_outer, 1);
      if (e == cudaSuccess) {
        // inner WHILE node in the outer body
        cudaStreamCaptureStatus status;
        cudaGraph_t g;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edges = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(s1, &status, nullptr, &g, &deps, &edges, &ndeps);
        if (e == cudaSuccess) {
          cudaGraphNodeParams np = {};
          np.type = cudaGraphNodeTypeConditional;
          np.conditional.handle = h_inner;
          np.conditional.type = cudaGraphCondTypeWhile;
          np.conditional.size = 1;
          cudaGraphNode_t node;
          e = cudaGraphAddNode(&node, g, deps, edges, ndeps, &np);
          if (e == cudaSuccess) {
            inner_body = np.conditional.phGraph_out[0];
            e = cudaStreamUpdateCaptureDependencies(s1, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
          }
        }
      }
      if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s2, inner_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        if (mixed) capture_pcg_iteration(p32, L, part, ctl, h_inner, s2);
        else capture_pcg_iteration(p64, L, part, ctl, h_inner, s2);
        cudaGraph_t tmp;
        e = cudaStreamEndCapture(s2, &tmp);
      }
      if (e == cudaSuccess) {
        if (mixed) {
          PIC_LAUNCH(G, kSB, 0, s1, k_axpy_out<float>)(L, x, p32.d, phi32, phi_c, dphi_dk);
        } else {
          PIC_LAUNCH(G, kSB, 0, s1, k_axpy_out<double>)(L, x, p64.d, nullptr, phi_c, dphi_dk);
        }
      }
      cudaGraph_t tmp1;
      cudaError_t e1 = cudaStreamEndCapture(s1, &tmp1);
      if (e == cudaSuccess) e = e1;
    }
    cudaGraph_t whole = nullptr;
    cudaError_t e0 = cudaStreamEndCapture(s0, &whole);
    if (e == cudaSuccess) e = e0;
    graph = whole;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaStreamDestroy(s0);
  cudaStreamDestroy(s1);
  cudaStreamDestroy(s2);
  if (e != cudaSuccess) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    cudaGetLastError();
  }
  return e;
}

cudaError_t Solver::launch(cudaStream_t s) {
  if (exec) {
    ++g_launches;
    return cudaGraphLaunch(exec, s);
  }
  return run_host(s);
}

// The same kernels driven from the host, one read-back per decision.
cudaError_t Solver::run_host(cudaStream_t s) {
  const Lv L = lv_of(plan[0]);
  const int G = sgrid(L.nu);
  const int mixed = precision != 0;
  const cudaGraphConditionalHandle none = 0;
  auto read = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(host_ctl, ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  };
  PIC_LAUNCH(G, kSB, 0, s, k_dot<double>)(L.nu, b, b, part);
  PIC_LAUNCH(1, kFinBlock, 0, s, k_fin_bb)(part, G, ctl, h_rtol, h_maxit);
  for (int outer = 0; outer < max_outer + 1; ++outer) {
    if (mixed) PIC_LAUNCH(G, kSB, 0, s, k_residual_prep<float>)(L, hx, b, p32.r, p32.d, part, ctl);
    else PIC_LAUNCH(G, kSB, 0, s, k_residual_prep<double>)(L, hx, b, p64.r, p64.d, part, ctl);
    PIC_LAUNCH(1, kFinBlock, 0, s, k_fin_outer)(part, G, ctl, none, none, inner_rtol, mixed, max_outer, 0);
    cudaError_t e = read();
    if (e != cudaSuccess) return e;
    const bool go = host_ctl->more != 0;
    while (go) {
      if (mixed) capture_pcg_iteration(p32, L, part, ctl, none, s, 0);
      else capture_pcg_iteration(p64, L, part, ctl, none, s, 0);
      if ((e = read()) != cudaSuccess) return e;
      if (!host_ctl->more) break;
    }
    if (mixed) PIC_LAUNCH(G, kSB, 0, s, k_axpy_out<float>)(L, hx, p32.d, hphi32, h_phi_c, h_dphi_dk);
    else PIC_LAUNCH(G, kSB, 0, s, k_axpy_out<double>)(L, hx, p64.d, nullptr, h_phi_c, h_dphi_dk);
    if (!go) break;
  }
  return cudaGetLastError();
}

SolveResult Solver::result(cudaStream_t s) {
  cudaMemcpyAsync(host_ctl, ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  SolveResult r;
  r.iters = host_ctl->it_total;
  r.resid_rel = host_ctl->resid_rel;
  r.converged = host_ctl->converged != 0;
  return r;
}

}  // namespace pic
