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

// x += alpha p ; r -= alpha q ; part = r . r
template <class T>
__global__ void __launch_bounds__(kSB) k_update(long long n, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                const T* __restrict__ q, const CgScalars* sc, double* part) {
  const T alpha = (T)sc->alpha;
  T acc = 0;
  for (long long u = gtid(); u < n; u += gstride()) {
    x[u] += alpha * p[u];
    const T rv = r[u] - alpha * q[u];
    r[u] = rv;
    acc += rv * rv;
  }
  block_partial<T, T>(acc, part);
}

// p = z + beta p
template <class T>
__global__ void __launch_bounds__(kSB) k_pupdate(long long n, T* __restrict__ p, const T* __restrict__ z, const CgScalars* sc) {
  const T beta = (T)sc->beta;
  for (long long u = gtid(); u < n; u += gstride()) p[u] = z[u] + beta * p[u];
}

// scalar updates from the block partials (single thread, fixed order)
enum { SC_RZ = 0, SC_PQ = 1, SC_RR = 2, SC_BB = 3 };
__global__ void k_scalars(const double* part, int nparts, int which, CgScalars* sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < nparts; ++i) s += part[i];
  if (which == SC_RZ) {
    sc->beta = sc->it > 0 ? s / sc->rz : 0.0;
    sc->rz = s;
  } else if (which == SC_PQ) {
    sc->pq = s;
    sc->alpha = s != 0.0 ? sc->rz / s : 0.0;
    sc->it += 1;
  } else if (which == SC_RR) {
    sc->rr = s;
  } else {
    sc->bb = s;
  }
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
    for (int c = 0; c < nk; ++c) {
      const int K = K0 + c;  // coarse node
      if (K <= 0 || K >= Cc.nz) continue;
      for (int b2 = 0; b2 < nj; ++b2) {
        const int J = (J0 + b2) % Cc.ny;
        for (int a2 = 0; a2 < ni; ++a2) {
          const int I = (I0 + a2) % Cc.nx;
          s += ec[(long long)(K - 1) * Cc.pl + (long long)J * Cc.nx + I];
        }
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
// PCG on level 0: x (in/out), b; vectors r, z, p, q (type T)
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
  if ((err = cudaMalloc(&part, sizeof(double) * kMaxRedBlocks))) return err;
  if ((err = cudaMalloc(&sc, sizeof(CgScalars)))) return err;
  if ((err = cudaMallocHost(&host_sc, sizeof(CgScalars)))) return err;
  return mg.init(plan);
}

template <class T>
void Pcg<T>::release() {
  cudaFree(r);
  cudaFree(z);
  cudaFree(p);
  cudaFree(q);
  cudaFree(part);
  cudaFree(sc);
  if (host_sc) cudaFreeHost(host_sc);
  host_sc = nullptr;
  mg.release();
}

template <class T>
double Pcg<T>::read_scalar(int which, cudaStream_t s) {
  cudaMemcpyAsync(host_sc, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return which == SC_RR ? host_sc->rr : host_sc->bb;
}

// Solve A x = b from the initial x until sqrt(r.r) <= tol_abs (recursive
// residual) or maxit; r must hold b - A x on entry and rr its squared norm.
template <class T>
int Pcg<T>::iterate(T* x, double rr0, double tol_abs, int maxit, cudaStream_t s, double* rr_out) {
  const Lv L = lv_of(mg.levels[0]);
  const int G = sgrid(n);
  CgScalars zero{};
  cudaMemcpyAsync(sc, &zero, sizeof(CgScalars), cudaMemcpyHostToDevice, s);
  double rr = rr0;
  int it = 0;
  while (std::sqrt(rr) > tol_abs && it < maxit) {
    mg.vcycle(r, z, s);
    PIC_LAUNCH(G, kSB, 0, s, k_dot<T>)(n, r, z, part);
    PIC_LAUNCH(1, 1, 0, s, k_scalars)(part, G, SC_RZ, sc);
    if (it == 0)
      PIC_LAUNCH(G, kSB, 0, s, k_copy<T>)(n, p, z);
    else
      PIC_LAUNCH(G, kSB, 0, s, k_pupdate<T>)(n, p, z, sc);
    PIC_LAUNCH(G, kSB, 0, s, k_apply_dot<T>)(L, p, q, part);
    PIC_LAUNCH(1, 1, 0, s, k_scalars)(part, G, SC_PQ, sc);
    PIC_LAUNCH(G, kSB, 0, s, k_update<T>)(n, x, r, p, q, sc, part);
    PIC_LAUNCH(1, 1, 0, s, k_scalars)(part, G, SC_RR, sc);
    rr = read_scalar(SC_RR, s);
    ++it;
    if (!std::isfinite(rr)) break;
  }
  *rr_out = rr;
  return it;
}

template struct Mg<double>;
template struct Mg<float>;
template struct Pcg<double>;
template struct Pcg<float>;

// ---------------------------------------------------------------------------
// Solver front ends
// ---------------------------------------------------------------------------
cudaError_t Solver::init(int nx, int ny, int nz, int precision_) {
  precision = precision_;
  plan = mg_plan(nx, ny, nz);
  n = plan[0].nu;
  cudaError_t err;
  if ((err = cudaMalloc(&b, sizeof(double) * (size_t)(n > 0 ? n : 1)))) return err;
  if ((err = cudaMalloc(&part, sizeof(double) * kMaxRedBlocks))) return err;
  if ((err = cudaMalloc(&sc, sizeof(CgScalars)))) return err;
  if ((err = cudaMallocHost(&host_sc, sizeof(CgScalars)))) return err;
  if (precision == 0) return p64.init(plan);
  if ((err = cudaMalloc(&r64, sizeof(double) * (size_t)(n > 0 ? n : 1)))) return err;
  if ((err = cudaMalloc(&d32, sizeof(float) * (size_t)(n > 0 ? n : 1)))) return err;
  return p32.init(plan);
}

void Solver::release() {
  cudaFree(b);
  cudaFree(part);
  cudaFree(sc);
  if (host_sc) cudaFreeHost(host_sc);
  host_sc = nullptr;
  cudaFree(r64);
  cudaFree(d32);
  p64.release();
  p32.release();
}

double Solver::reduce_host(int G, cudaStream_t s) {
  PIC_LAUNCH(1, 1, 0, s, k_scalars)(part, G, SC_BB, sc);
  cudaMemcpyAsync(host_sc, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return host_sc->bb;
}

// x: unknown-node view of phi (nodes k = 1..nz-1, contiguous); b must be set.
SolveResult Solver::solve(double* x, double rtol, int maxit, cudaStream_t s) {
  SolveResult res{0, 0.0, true};
  const Lv L = lv_of(plan[0]);
  const int G = sgrid(n);
  if (n == 0) return res;
  PIC_LAUNCH(G, kSB, 0, s, k_dot<double>)(n, b, b, part);
  const double bb = reduce_host(G, s);
  if (bb == 0.0) {
    PIC_LAUNCH(G, kSB, 0, s, k_zero<double>)(n, x);
    return res;
  }
  const double tol = rtol * std::sqrt(bb);
  int total = 0;
  double rr_true = 0.0;
  if (precision == 0) {
    for (int restart = 0; restart < 8; ++restart) {
      PIC_LAUNCH(G, kSB, 0, s, k_residual<double, double>)(L, x, b, p64.r, part);
      const double rr = reduce_host(G, s);
      rr_true = rr;
      if (std::sqrt(rr) <= tol || total >= maxit) break;
      double rr_end = 0.0;
      total += p64.iterate(x, rr, tol, maxit - total, s, &rr_end);
      if (!std::isfinite(rr_end)) break;
    }
  } else {
    // iterative refinement: FP64 residual and update, FP32 correction solve
    for (int outer = 0; outer < 40; ++outer) {
      PIC_LAUNCH(G, kSB, 0, s, k_residual<double, double>)(L, x, b, r64, part);
      const double rr = reduce_host(G, s);
      rr_true = rr;
      if (std::sqrt(rr) <= tol || total >= maxit || !std::isfinite(rr)) break;
      // r32 = r64, d = 0; inner PCG on A d = r to inner_rtol relative
      PIC_LAUNCH(G, kSB, 0, s, k_copy_cast)(n, p32.r, r64);
      PIC_LAUNCH(G, kSB, 0, s, k_zero<float>)(n, d32);
      double rr_end = 0.0;
      const double tol_in = std::max(inner_rtol * std::sqrt(rr), 0.5 * tol);
      total += p32.iterate(d32, rr, tol_in, maxit - total, s, &rr_end);
      PIC_LAUNCH(G, kSB, 0, s, k_axpy_cast<float>)(n, x, d32);
    }
  }
  res.iters = total;
  res.resid_rel = std::sqrt(rr_true / bb);
  res.converged = res.resid_rel <= rtol;
  return res;
}


}  // namespace pic
