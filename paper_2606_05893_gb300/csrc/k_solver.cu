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
#include <type_traits>
#include <utility>

#include <cooperative_groups.h>
#include <vector>

#include "dev_mem.cuh"
#include "pic_internal.cuh"
#include "pic_kernels.cuh"
#include "tc_ptx.cuh"
#include "pic_solver.cuh"

namespace pic {

// Programmatic dependent launch: each solver kernel may be launched while its
// predecessor drains (it waits here until the predecessor has completed and its
// writes are visible), and lets its own successor launch as soon as all of its
// blocks are running. Hides most of the launch gap between the many short
// multigrid kernels. A no-op for kernels launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

bool g_pdl = true;  // cleared when a graph with programmatic edges cannot be built

template <class K>
struct PdlLaunch {
  K k;
  dim3 g, b;
  size_t smem;
  cudaStream_t s;
  template <class... A>
  void operator()(A&&... a) const {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = g_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(a)...);
  }
};
#define SOLVER_LAUNCH(grid, block, smem, stream, ...) \
  (::pic::count_kernel()), ::pic::PdlLaunch<decltype(&__VA_ARGS__)>{&__VA_ARGS__, dim3(grid), dim3(block), (size_t)(smem), stream}

constexpr int kSB = 256;
constexpr int kMaxRedBlocks = 152 * 8;  // 1-D reductions over whole vectors
constexpr int kPartsMax = 1 << 16;      // capacity of the block-partials buffer
constexpr int kPlaneBlocks = 8;         // blocks per plane in plane-major kernels

static int sgrid(long long n) {
  long long b = (n + kSB - 1) / kSB;
  if (b < 1) b = 1;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
  return (int)b;
}

// Level geometry with 32-bit indices (a level holds far fewer than 2^31 unknowns).
struct Lv {
  int nx, ny, nz, pl, nu;
};
static Lv lv_of(const MgLevel& L) { return Lv{L.nx, L.ny, L.nz, L.nx * L.ny, (int)L.nu}; }

// 3-D launches without integer division (on GB300 int division and int<->float
// conversions run on the narrow FP64/conversion pipe): block (32, 8); x covers
// the `xe` points of a row, y strides over the rows j, z = unknown plane.
constexpr int kBX = 32, kBY = 8, kMaxGY = 4;
static dim3 g3(const Lv& L, int xe) {
  int gy = (L.ny + kBY - 1) / kBY;
  gy = gy > kMaxGY ? kMaxGY : gy;
  return dim3((xe + kBX - 1) / kBX, gy, L.nz - 1 > 0 ? L.nz - 1 : 1);
}
static const dim3 kB3(kBX, kBY, 1);

template <class T>
__device__ __forceinline__ T nb_sum(const Lv& L, const T* __restrict__ x, int u, int i, int j, int k) {
  // k: unknown plane index 0..nz-2
  const int row = u - i;
  const int im = i == 0 ? L.nx - 1 : i - 1, ip = i == L.nx - 1 ? 0 : i + 1;
  const int rm = j == 0 ? (L.ny - 1) * L.nx : -L.nx;
  const int rp = j == L.ny - 1 ? -(L.ny - 1) * L.nx : L.nx;
  T s = x[row + im] + x[row + ip] + x[u + rm] + x[u + rp];
  if (k > 0) s += x[u - L.pl];
  if (k < L.nz - 2) s += x[u + L.pl];
  return s;
}

// loop header of the 3-D kernels: i over [0, xe), j over the rows, k = plane
#define ROWS3(L, xe)                                                          \
  const int k = blockIdx.z;                                                  \
  const int i = blockIdx.x * kBX + threadIdx.x;                              \
  const bool in_x = i < (xe);                                                \
  for (int j = blockIdx.y * kBY + threadIdx.y; j < (L).ny; j += gridDim.y * kBY)

// The same with k striding over the planes too, for the kernels that end in a
// grid-wide sum: launched on g3r (at most one wave of blocks), so each block
// pays the partial's fence and ticket once for several planes.
#define ROWS3K(L, xe)                                                         \
  const int i = blockIdx.x * kBX + threadIdx.x;                              \
  const bool in_x = i < (xe);                                                \
  for (int k = blockIdx.z; k < (L).nz - 1; k += gridDim.z)                   \
    for (int j = blockIdx.y * kBY + threadIdx.y; j < (L).ny; j += gridDim.y * kBY)
constexpr int kWaveBlocks = 152 * 8;  // resident 256-thread blocks on 152 SMs
static dim3 g3rs(const Lv& L) {  // as g3r, x over the nx / 2 points of a colour
  dim3 g = g3(L, L.nx / 2);
  const int per_plane = (int)(g.x * g.y);
  int gz = kWaveBlocks / per_plane;
  gz = gz < 1 ? 1 : (gz > (int)g.z ? (int)g.z : gz);
  g.z = gz;
  return g;
}
static dim3 g3r(const Lv& L) {
  dim3 g = g3(L, L.nx);
  const int per_plane = (int)(g.x * g.y);
  int gz = kWaveBlocks / per_plane;
  gz = gz < 1 ? 1 : (gz > (int)g.z ? (int)g.z : gz);
  g.z = gz;
  return g;
}

// r = b - A x at the colour-0 points only (x index m over the nx/2 points of
// that colour, as the half sweeps). After the pre-smoothing half sweeps the
// colour-1 residual is zero in exact arithmetic (the colour-1 sweep solved
// those equations with their colour-0 neighbours fixed), so it is neither
// formed nor restricted; the V-cycle is the same operator.
template <class T>
__global__ void __launch_bounds__(256) k_residual(Lv L, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r) {
  pdl_enter();
  const int m = blockIdx.x * kBX + threadIdx.x;
  const int k = blockIdx.z;
  if (m >= (L.nx >> 1)) return;
  for (int j = blockIdx.y * kBY + threadIdx.y; j < L.ny; j += gridDim.y * kBY) {
    const int i = 2 * m + ((j + k + 1) & 1);
    const int u = k * L.pl + j * L.nx + i;
    r[u] = b[u] - ((T)6 * x[u] - nb_sum(L, x, u, i, j, k));
  }
}

// ---------------------------------------------------------------------------
// multigrid pieces
// ---------------------------------------------------------------------------
// One red-black Gauss-Seidel half sweep: points with (i + j + knode) % 2 == color
// (x index m covers the nx/2 points of that colour in a row).
template <class T>
__global__ void __launch_bounds__(256) k_smooth(Lv L, T* __restrict__ e, const T* __restrict__ b, int color) {
  pdl_enter();
  const T sixth = (T)(1.0 / 6.0);
  const int hx = L.nx >> 1;
  const int m = blockIdx.x * kBX + threadIdx.x;
  const int k = blockIdx.z;
  if (m >= hx) return;
  for (int j = blockIdx.y * kBY + threadIdx.y; j < L.ny; j += gridDim.y * kBY) {
    const int i = 2 * m + ((j + k + 1 + color) & 1);
    const int u = k * L.pl + j * L.nx + i;
    e[u] = (b[u] + nb_sum(L, e, u, i, j, k)) * sixth;
  }
}

// products rounded on their own (no contraction into a neighbouring add), so a
// value recomputed in a register equals the one a separate kernel stored
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// nb_sum of the values x / 6 (each product rounded as a stored x / 6 would be)
template <class T>
__device__ __forceinline__ T nb_sum_sixth(const Lv& L, const T* __restrict__ x, int u, int i, int j, int k, T sixth) {
  const int row = u - i;
  const int im = i == 0 ? L.nx - 1 : i - 1, ip = i == L.nx - 1 ? 0 : i + 1;
  const int rm = j == 0 ? (L.ny - 1) * L.nx : -L.nx;
  const int rp = j == L.ny - 1 ? -(L.ny - 1) * L.nx : L.nx;
  T s = mul_rn(x[row + im], sixth) + mul_rn(x[row + ip], sixth) + mul_rn(x[u + rm], sixth) + mul_rn(x[u + rp], sixth);
  if (k > 0) s += mul_rn(x[u - L.pl], sixth);
  if (k < L.nz - 2) s += mul_rn(x[u + L.pl], sixth);
  return s;
}

// The two pre-smoothing half sweeps from e = 0 in one pass: colour 0 takes
// b / 6, colour 1 then takes (b + the sum of its colour-0 neighbours) / 6, the
// neighbours' b / 6 recomputed here. Same values as the two sweeps.
template <class T>
__global__ void __launch_bounds__(256) k_smooth_pre(Lv L, T* __restrict__ e, const T* __restrict__ b) {
  pdl_enter();
  const T sixth = (T)(1.0 / 6.0);
  const int hx = L.nx >> 1;
  const int m = blockIdx.x * kBX + threadIdx.x;
  const int k = blockIdx.z;
  if (m >= hx) return;
  for (int j = blockIdx.y * kBY + threadIdx.y; j < L.ny; j += gridDim.y * kBY) {
    const int par = (j + k + 1) & 1;  // colour 0 at i = 2m + par
    const int i0 = 2 * m + par, i1 = 2 * m + (par ^ 1);
    const int row = k * L.pl + j * L.nx;
    e[row + i0] = mul_rn(b[row + i0], sixth);
    e[row + i1] = (b[row + i1] + nb_sum_sixth(L, b, row + i1, i1, j, k, sixth)) * sixth;
  }
}

// b_c = 4 * full-weighting(r_f) on coarse unknowns (grid over the coarse level)
template <class T>
__global__ void __launch_bounds__(256) k_restrict(Lv F, Lv Cc, const T* __restrict__ r, T* __restrict__ bc) {
  pdl_enter();
  const int I = blockIdx.x * kBX + threadIdx.x;
  const int K = blockIdx.z;
  if (I >= Cc.nx) return;
  const int Kn = K + 1;  // coarse node index
  const int i0 = 2 * I;
  const int im = i0 == 0 ? F.nx - 1 : i0 - 1;
  const int ip = i0 + 1 == F.nx ? 0 : i0 + 1;
  for (int J = blockIdx.y * kBY + threadIdx.y; J < Cc.ny; J += gridDim.y * kBY) {
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
        const int rowf = kf * F.pl + jf * F.nx;
        // colour-0 fine points only (even offset sum; the colour-1 residual is zero)
        if (((b2 + c) & 1) == 0) s += wb * wc * ((T)0.5 * r[rowf + i0]);
        else s += wb * wc * ((T)0.25 * (r[rowf + im] + r[rowf + ip]));
      }
    }
    bc[K * Cc.pl + J * Cc.nx + I] = (T)4 * s;
  }
}

// e_f += P e_c (trilinear; coarse Dirichlet planes carry 0) on the colour-0
// points only: the colour-1 half sweep that follows reads colour-0 neighbours
// alone and overwrites colour 1, so prolonged colour-1 values would never be
// read. Grid as for the half sweeps (x covers the nx / 2 points of a colour).
template <class T>
__global__ void __launch_bounds__(256) k_prolong(Lv F, Lv Cc, const T* __restrict__ ec, T* __restrict__ ef) {
  pdl_enter();
  const int kn = blockIdx.z + 1;  // fine node plane
  const int K0 = kn >> 1;
  const bool kodd = kn & 1;
  const bool use0 = K0 >= 1 && K0 <= Cc.nz - 1;
  const bool use1 = kodd && (K0 + 1) >= 1 && (K0 + 1) <= Cc.nz - 1;
  const int off0 = (K0 - 1) * Cc.pl, off1 = K0 * Cc.pl;
  const T wk = kodd ? (T)0.5 : (T)1;
  const int m = blockIdx.x * kBX + threadIdx.x;
  if (m >= (F.nx >> 1)) return;
  for (int j = blockIdx.y * kBY + threadIdx.y; j < F.ny; j += gridDim.y * kBY) {
    const int i = 2 * m + ((j + (int)blockIdx.z + 1) & 1);  // colour 0
    const int I0 = i >> 1;
    const int I1 = I0 + 1 == Cc.nx ? 0 : I0 + 1;
    const bool iodd = i & 1;
    const int J0 = j >> 1;
    const int J1 = J0 + 1 == Cc.ny ? 0 : J0 + 1;
    const bool jodd = j & 1;
    T s = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c == 0 ? !use0 : !use1) continue;
      const int off = c == 0 ? off0 : off1;
      const int r0 = off + J0 * Cc.nx, r1 = off + J1 * Cc.nx;
      T t = ec[r0 + I0];
      if (iodd) t = (T)0.5 * (t + ec[r0 + I1]);
      if (jodd) {
        T t1 = ec[r1 + I0];
        if (iodd) t1 = (T)0.5 * (t1 + ec[r1 + I1]);
        t = (T)0.5 * (t + t1);
      }
      s += t;
    }
    ef[blockIdx.z * F.pl + j * F.nx + i] += wk * s;
  }
}

// ---------------------------------------------------------------------------
// Colour-split layout of the finest level (MIXED path): every colour-0 point,
// then every colour-1 point, each half in (plane, row, m) order with m = i / 2.
// A half sweep in the natural order reads one colour with stride 2 (a warp's
// load spans twice the bytes it uses); here every neighbour a point needs is a
// contiguous run of the other colour: its y and z neighbours sit at the same m,
// its x neighbours at m - 1 + p and m + p (p = the parity of i, (j + k + 1 + c)
// & 1 for colour c; nx, ny even). The sums keep the natural kernels' order, so
// the values are theirs.
// ---------------------------------------------------------------------------
template <class V>
__device__ __forceinline__ bool grid_total(V v, double* part, unsigned* ticket, double* tot);
__device__ __forceinline__ void set_beta(SolveCtl* c, double rz);

struct SpNb {
  int xm, xp, ym, yp, zm, zp;  // offsets into the other colour's half (zm / zp: -1 when absent)
};
// neighbours of point (m, j, k) of parity p in the other colour's half
__device__ __forceinline__ SpNb sp_nb(const Lv& L, int m, int j, int k, int p) {
  const int hx = L.nx >> 1;
  const int row = (k * L.ny + j) * hx;
  SpNb n;
  int a = m - 1 + p, b = m + p;
  a = a < 0 ? hx - 1 : a;
  b = b == hx ? 0 : b;
  n.xm = row + a;
  n.xp = row + b;
  n.ym = (j == 0 ? row + (L.ny - 1) * hx : row - hx) + m;
  n.yp = (j == L.ny - 1 ? row - (L.ny - 1) * hx : row + hx) + m;
  n.zm = k > 0 ? row - L.ny * hx + m : -1;
  n.zp = k < L.nz - 2 ? row + L.ny * hx + m : -1;
  return n;
}
template <class T>
__device__ __forceinline__ T sp_sum(const T* __restrict__ o, const SpNb& n) {
  T s = o[n.xm] + o[n.xp] + o[n.ym] + o[n.yp];
  if (n.zm >= 0) s += o[n.zm];
  if (n.zp >= 0) s += o[n.zp];
  return s;
}
template <class T>
__device__ __forceinline__ T sp_sum_sixth(const T* __restrict__ o, const SpNb& n, T sixth) {
  T s = mul_rn(o[n.xm], sixth) + mul_rn(o[n.xp], sixth) + mul_rn(o[n.ym], sixth) + mul_rn(o[n.yp], sixth);
  if (n.zm >= 0) s += mul_rn(o[n.zm], sixth);
  if (n.zp >= 0) s += mul_rn(o[n.zp], sixth);
  return s;
}
// split index of natural point (i, j, k)
__device__ __forceinline__ int sp_index(const Lv& L, int i, int j, int k) {
  const int hx = L.nx >> 1;
  return ((i + j + k + 1) & 1) * (L.nu >> 1) + (k * L.ny + j) * hx + (i >> 1);
}

// the loop header of the split kernels: m over the nx / 2 points of a colour in
// a row, j over the rows, k = plane (grid g3(L, nx / 2))
#define SPLIT_ROWS(L)                                                        \
  const int m = blockIdx.x * kBX + threadIdx.x;                              \
  const int k = blockIdx.z;                                                  \
  const int hx_ = (L).nx >> 1;                                               \
  const int half_ = (L).nu >> 1;                                             \
  if (m >= hx_) return;                                                      \
  for (int j = blockIdx.y * kBY + threadIdx.y; j < (L).ny; j += gridDim.y * kBY)

template <class T>
__global__ void __launch_bounds__(256) k_smooth_s(Lv L, T* __restrict__ e, const T* __restrict__ b, int color) {
  pdl_enter();
  const T sixth = (T)(1.0 / 6.0);
  SPLIT_ROWS(L) {
    const int p = (j + k + 1 + color) & 1;
    const int u = color * half_ + (k * L.ny + j) * hx_ + m;
    const SpNb n = sp_nb(L, m, j, k, p);
    e[u] = (b[u] + sp_sum(e + (color ^ 1) * half_, n)) * sixth;
  }
}

// The V-cycle's last half sweep (colour 0 of the split finest level) with the
// PCG product r.z: each thread adds its colour-0 point, just written, and the
// colour-1 point at the same index of the other half, final since the sweep
// before; the last block turns r.z into beta. Planes strided on at most one
// wave of blocks (every thread reaches the grid-wide sum).
template <class T>
__global__ void __launch_bounds__(256) k_smooth_s_dot(Lv L, T* __restrict__ e, const T* __restrict__ b, double* part,
                                                      SolveCtl* c) {
  pdl_enter();
  const T sixth = (T)(1.0 / 6.0);
  const int m = blockIdx.x * kBX + threadIdx.x;
  const int hx = L.nx >> 1, half = L.nu >> 1;
  T acc = 0;
  if (m < hx) {
    for (int k = blockIdx.z; k < L.nz - 1; k += gridDim.z)
      for (int j = blockIdx.y * kBY + threadIdx.y; j < L.ny; j += gridDim.y * kBY) {
        const int u = (k * L.ny + j) * hx + m;
        const SpNb n = sp_nb(L, m, j, k, (j + k + 1) & 1);
        const T b0 = b[u];
        const T e0 = (b0 + sp_sum(e + half, n)) * sixth;
        e[u] = e0;
        acc += b0 * e0 + b[half + u] * e[half + u];
      }
  }
  double rz;
  if (grid_total(acc, part, &c->ticket, &rz)) set_beta(c, rz);
}

template <class T>
__global__ void __launch_bounds__(256) k_smooth_pre_s(Lv L, T* __restrict__ e, const T* __restrict__ b) {
  pdl_enter();
  const T sixth = (T)(1.0 / 6.0);
  SPLIT_ROWS(L) {
    const int u = (k * L.ny + j) * hx_ + m;
    e[u] = mul_rn(b[u], sixth);  // colour 0 from e = 0
    const SpNb n = sp_nb(L, m, j, k, (j + k) & 1);  // colour 1, its neighbours colour 0
    e[half_ + u] = (b[half_ + u] + sp_sum_sixth(b, n, sixth)) * sixth;
  }
}

// residual at the colour-0 points (written into the colour-0 half)
template <class T>
__global__ void __launch_bounds__(256) k_residual_s(Lv L, const T* __restrict__ x, const T* __restrict__ b,
                                                    T* __restrict__ r) {
  pdl_enter();
  SPLIT_ROWS(L) {
    const int u = (k * L.ny + j) * hx_ + m;
    const SpNb n = sp_nb(L, m, j, k, (j + k + 1) & 1);
    r[u] = b[u] - ((T)6 * x[u] - sp_sum(x + half_, n));
  }
}

// b_c = 4 * full-weighting of the colour-0 residual of the split finest level
// (natural coarse output; grid over the coarse level). The colour-0 points of
// the 27-point stencil have an even offset sum: the centre column (i = 2I) when
// the row and plane offsets sum to an even number, else its two x-neighbours
// (i = 2I +- 1, both of m = I and I - 1).
template <class T>
__global__ void __launch_bounds__(256) k_restrict_s0(Lv F, Lv Cc, const T* __restrict__ r, T* __restrict__ bc) {
  pdl_enter();
  const int I = blockIdx.x * kBX + threadIdx.x;
  const int K = blockIdx.z;
  if (I >= Cc.nx) return;
  const int Kn = K + 1;
  const int hx = F.nx >> 1;
  const int Im = I == 0 ? hx - 1 : I - 1;
  for (int J = blockIdx.y * kBY + threadIdx.y; J < Cc.ny; J += gridDim.y * kBY) {
    T s = 0;
#pragma unroll
    for (int c = -1; c <= 1; ++c) {
      const int kf = 2 * Kn + c - 1;
      const T wc = c == 0 ? (T)0.5 : (T)0.25;
#pragma unroll
      for (int b2 = -1; b2 <= 1; ++b2) {
        int jf = 2 * J + b2;
        jf = jf < 0 ? jf + F.ny : (jf >= F.ny ? jf - F.ny : jf);
        const T wb = b2 == 0 ? (T)0.5 : (T)0.25;
        const int rowf = (kf * F.ny + jf) * hx;
        if (((b2 + c) & 1) == 0) s += wb * wc * ((T)0.5 * r[rowf + I]);
        else s += wb * wc * ((T)0.25 * (r[rowf + Im] + r[rowf + I]));
      }
    }
    bc[K * Cc.pl + J * Cc.nx + I] = (T)4 * s;
  }
}

// e_f += P e_c at the colour-0 points of the split finest level (natural coarse input)
template <class T>
__global__ void __launch_bounds__(256) k_prolong_s0(Lv F, Lv Cc, const T* __restrict__ ec, T* __restrict__ ef) {
  pdl_enter();
  const int kn = blockIdx.z + 1;
  const int K0 = kn >> 1;
  const bool kodd = kn & 1;
  const bool use0 = K0 >= 1 && K0 <= Cc.nz - 1;
  const bool use1 = kodd && (K0 + 1) >= 1 && (K0 + 1) <= Cc.nz - 1;
  const int off0 = (K0 - 1) * Cc.pl, off1 = K0 * Cc.pl;
  const T wk = kodd ? (T)0.5 : (T)1;
  const int m = blockIdx.x * kBX + threadIdx.x;
  const int hx = F.nx >> 1;
  if (m >= hx) return;
  const int I0 = m;  // i >> 1 for both parities
  const int I1 = I0 + 1 == Cc.nx ? 0 : I0 + 1;
  for (int j = blockIdx.y * kBY + threadIdx.y; j < F.ny; j += gridDim.y * kBY) {
    const bool iodd = ((j + (int)blockIdx.z + 1) & 1) != 0;  // parity of i at colour 0
    const int J0 = j >> 1;
    const int J1 = J0 + 1 == Cc.ny ? 0 : J0 + 1;
    const bool jodd = j & 1;
    T s = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c == 0 ? !use0 : !use1) continue;
      const int off = c == 0 ? off0 : off1;
      const int r0 = off + J0 * Cc.nx, r1 = off + J1 * Cc.nx;
      T t = ec[r0 + I0];
      if (iodd) t = (T)0.5 * (t + ec[r0 + I1]);
      if (jodd) {
        T t1 = ec[r1 + I0];
        if (iodd) t1 = (T)0.5 * (t1 + ec[r1 + I1]);
        t = (T)0.5 * (t + t1);
      }
      s += t;
    }
    ef[(blockIdx.z * F.ny + j) * hx + m] += wk * s;
  }
}

template <class T>
__global__ void k_coarse(long long n, const T* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ e) {
  pdl_enter();
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
  pdl_enter();
  for (long long u = gtid(); u < n; u += gstride()) x[u] += (double)d[u];
}
template <class T>
__global__ void k_zero(long long n, T* __restrict__ x) {
  pdl_enter();
  for (long long u = gtid(); u < n; u += gstride()) x[u] = (T)0;
}
template <class T>
__global__ void k_copy(long long n, T* __restrict__ d, const T* __restrict__ s) {
  pdl_enter();
  for (long long u = gtid(); u < n; u += gstride()) d[u] = s[u];
}

__global__ void k_copy_cast(long long n, float* __restrict__ d, const double* __restrict__ s) {
  pdl_enter();
  for (long long u = gtid(); u < n; u += gstride()) d[u] = (float)s[u];
}
template <class T>
__global__ void k_jacobi_scale(long long n, T* z) {
  pdl_enter();
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

// ---------------------------------------------------------------------------
// The deepest multigrid levels in one thread-block cluster (FP32). Launch
// latency, not bandwidth, bounds the small levels: about 20 dependent kernels
// of a few microseconds each per V-cycle. Here 8 blocks of one cluster hold the
// levels in shared memory, split by unknown planes (block c owns planes
// [c P / 8, (c + 1) P / 8) of every level), read neighbouring planes owned by
// other blocks through distributed shared memory, and separate the phases
// with cluster barriers; the operations are those of the per-level kernels.
// Every thread of every block passes every barrier (no early exit).
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;
constexpr int kClusterCTAs = 8;
constexpr int kClusterThreads = 1024;
constexpr int kMaxFused = 6;
constexpr int kMaxPlanes = 128;  // unknown planes of a fused level
constexpr long long kClusterMaxUnknowns = 16384;

struct KLv {
  int nx, ny, P, pl, hx;  // cells x, y; unknown planes; plane size; nx / 2
  FastDiv dnx, dpl, dhx, dhxny;
  int maxp;               // planes per block at most
  int oe, ob, orr;        // shared-memory offsets (floats) of e, b, r (maxp planes each)
};
struct ClusterArgs {
  int nlev;  // fused levels, the last the coarsest
  KLv L[kMaxFused];
  int dense, nuc, ocb;  // coarsest: dense inverse (nuc x nuc, global), local copy of its b at ocb
  int coarse_sweeps;
  const float* Ainv;
  const float* b_in;  // b of the first fused level (global, all planes)
  float* e_out;       // e of the first fused level (global)
};

__device__ __forceinline__ int plane0(int P, int c) { return (c * P) / kClusterCTAs; }

// owner block and local index of every unknown plane of every fused level,
// built once per launch (no division in the phases)
struct PlaneMap {
  unsigned char own[kMaxFused][kMaxPlanes];
  unsigned char loc[kMaxFused][kMaxPlanes];
};

// pointer to plane k of an array (offset off) of level l, local or in another block
__device__ __forceinline__ float* plane_ptr(float* sm, const PlaneMap& pm, int l, const KLv& L, int off, int k,
                                            int me) {
  const int o = pm.own[l][k];
  float* base = sm + off + pm.loc[l][k] * L.pl;
  return o == me ? base : static_cast<float*>(__cluster_map_shared_rank(base, o));
}

// sum of the six neighbours of (i, j) in plane k (local pointer c), planes k +- 1 via DSMEM
__device__ __forceinline__ float k_nb(float* sm, const PlaneMap& pm, int l, const KLv& L, int off, const float* c,
                                      int k, int i, int j, int me) {
  const int im = i == 0 ? L.nx - 1 : i - 1, ip = i == L.nx - 1 ? 0 : i + 1;
  const int jm = j == 0 ? L.ny - 1 : j - 1, jp = j == L.ny - 1 ? 0 : j + 1;
  const int r = j * L.nx;
  float s = c[r + im] + c[r + ip] + c[jm * L.nx + i] + c[jp * L.nx + i];
  if (k > 0) s += plane_ptr(sm, pm, l, L, off, k - 1, me)[r + i];
  if (k < L.P - 1) s += plane_ptr(sm, pm, l, L, off, k + 1, me)[r + i];
  return s;
}

__device__ void kc_smooth(float* sm, const PlaneMap& pm, int l, const KLv& L, int me, int color) {
  const float sixth = 1.0f / 6.0f;
  const int p0 = plane0(L.P, me), np = plane0(L.P, me + 1) - p0;
  const int per = L.hx * L.ny;
  for (int q = threadIdx.x; q < np * per; q += blockDim.x) {
    const int kk = fdiv(q, L.dhxny);
    const int t = q - kk * per;
    const int j = fdiv(t, L.dhx);
    const int m = t - j * L.hx;
    const int k = p0 + kk;
    const int i = 2 * m + ((j + k + 1 + color) & 1);
    float* e = sm + L.oe + kk * L.pl;
    const float* b = sm + L.ob + kk * L.pl;
    const int u = j * L.nx + i;
    e[u] = (b[u] + k_nb(sm, pm, l, L, L.oe, e, k, i, j, me)) * sixth;
  }
}

// the two pre-smoothing half sweeps from e = 0 in one phase (as k_smooth_pre)
__device__ void kc_smooth_pre(float* sm, const PlaneMap& pm, int l, const KLv& L, int me) {
  const float sixth = 1.0f / 6.0f;
  const int p0 = plane0(L.P, me), np = plane0(L.P, me + 1) - p0;
  const int per = L.hx * L.ny;
  for (int q = threadIdx.x; q < np * per; q += blockDim.x) {
    const int kk = fdiv(q, L.dhxny);
    const int t = q - kk * per;
    const int j = fdiv(t, L.dhx);
    const int m = t - j * L.hx;
    const int k = p0 + kk;
    const int par = (j + k + 1) & 1;
    const int i0 = 2 * m + par, i1 = 2 * m + (par ^ 1);
    float* e = sm + L.oe + kk * L.pl;
    const float* bp = sm + L.ob + kk * L.pl;
    const int r = j * L.nx;
    e[r + i0] = __fmul_rn(bp[r + i0], sixth);
    // colour-0 neighbours of (i1, j, k), each b / 6, summed in k_nb's order
    const int im = i1 == 0 ? L.nx - 1 : i1 - 1, ip = i1 == L.nx - 1 ? 0 : i1 + 1;
    const int jm = j == 0 ? L.ny - 1 : j - 1, jp = j == L.ny - 1 ? 0 : j + 1;
    float sn = __fmul_rn(bp[r + im], sixth) + __fmul_rn(bp[r + ip], sixth) + __fmul_rn(bp[jm * L.nx + i1], sixth) +
               __fmul_rn(bp[jp * L.nx + i1], sixth);
    if (k > 0) sn += __fmul_rn(plane_ptr(sm, pm, l, L, L.ob, k - 1, me)[r + i1], sixth);
    if (k < L.P - 1) sn += __fmul_rn(plane_ptr(sm, pm, l, L, L.ob, k + 1, me)[r + i1], sixth);
    e[r + i1] = (bp[r + i1] + sn) * sixth;
  }
}

// colour-0 points only, as k_residual
__device__ void kc_residual(float* sm, const PlaneMap& pm, int l, const KLv& L, int me) {
  const int p0 = plane0(L.P, me), np = plane0(L.P, me + 1) - p0;
  const int per = L.hx * L.ny;
  for (int q = threadIdx.x; q < np * per; q += blockDim.x) {
    const int kk = fdiv(q, L.dhxny);
    const int t = q - kk * per;
    const int j = fdiv(t, L.dhx);
    const int i = 2 * (t - j * L.hx) + ((j + p0 + kk + 1) & 1);
    const int u = j * L.nx + i;
    const float* e = sm + L.oe + kk * L.pl;
    sm[L.orr + kk * L.pl + u] =
        sm[L.ob + kk * L.pl + u] - (6.f * e[u] - k_nb(sm, pm, l, L, L.oe, e, p0 + kk, i, j, me));
  }
}

__device__ void kc_restrict(float* sm, const PlaneMap& pm, int l, const KLv& F, const KLv& C, int me) {
  const int p0 = plane0(C.P, me), np = plane0(C.P, me + 1) - p0;
  for (int q = threadIdx.x; q < np * C.pl; q += blockDim.x) {
    const int kk = fdiv(q, C.dpl);
    const int U = q - kk * C.pl;
    const int J = fdiv(U, C.dnx);
    const int I = U - J * C.nx;
    const int Kn = p0 + kk + 1;  // coarse node plane
    const int i0 = 2 * I;
    const int im = i0 == 0 ? F.nx - 1 : i0 - 1;
    const int ip = i0 + 1 == F.nx ? 0 : i0 + 1;
    float s = 0.f;
#pragma unroll
    for (int cc = -1; cc <= 1; ++cc) {
      const int kf = 2 * Kn + cc - 1;  // fine unknown plane
      const float wc = cc == 0 ? 0.5f : 0.25f;
      const float* rp = plane_ptr(sm, pm, l, F, F.orr, kf, me);
#pragma unroll
      for (int b2 = -1; b2 <= 1; ++b2) {
        int jf = 2 * J + b2;
        jf = jf < 0 ? jf + F.ny : (jf >= F.ny ? jf - F.ny : jf);
        const float wb = b2 == 0 ? 0.5f : 0.25f;
        const float* row = rp + jf * F.nx;
        if (((b2 + cc) & 1) == 0) s += wb * wc * (0.5f * row[i0]);
        else s += wb * wc * (0.25f * (row[im] + row[ip]));
      }
    }
    sm[C.ob + kk * C.pl + U] = 4.f * s;
  }
}

__device__ void kc_prolong(float* sm, const PlaneMap& pm, int l, const KLv& F, const KLv& C, int me) {
  // colour-0 points only (the colour-1 half sweep that follows reads colour 0 alone)
  const int p0 = plane0(F.P, me), np = plane0(F.P, me + 1) - p0;
  const int per = F.hx * F.ny;
  for (int q = threadIdx.x; q < np * per; q += blockDim.x) {
    const int kk = fdiv(q, F.dhxny);
    const int t = q - kk * per;
    const int j = fdiv(t, F.dhx);
    const int i = 2 * (t - j * F.hx) + ((j + p0 + kk + 1) & 1);
    const int u = j * F.nx + i;
    const int kn = p0 + kk + 1;  // fine node plane
    const int K0 = kn >> 1;
    const bool kodd = kn & 1;
    const int I0 = i >> 1;
    const int I1 = I0 + 1 == C.nx ? 0 : I0 + 1;
    const bool iodd = i & 1;
    const int J0 = j >> 1;
    const int J1 = J0 + 1 == C.ny ? 0 : J0 + 1;
    const bool jodd = j & 1;
    float s = 0.f;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int Kc = K0 + cc;  // coarse node plane
      if (cc == 1 && !kodd) continue;
      if (Kc < 1 || Kc > C.P) continue;
      const float* ep = plane_ptr(sm, pm, l + 1, C, C.oe, Kc - 1, me);
      const int r0 = J0 * C.nx, r1 = J1 * C.nx;
      float t = ep[r0 + I0];
      if (iodd) t = 0.5f * (t + ep[r0 + I1]);
      if (jodd) {
        float t1 = ep[r1 + I0];
        if (iodd) t1 = 0.5f * (t1 + ep[r1 + I1]);
        t = 0.5f * (t + t1);
      }
      s += t;
    }
    sm[F.oe + kk * F.pl + u] += kodd ? 0.5f * s : s;
  }
}

__global__ void __launch_bounds__(kClusterThreads) k_coarse_cluster(ClusterArgs a) {
  pdl_enter();
  extern __shared__ float sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int me = (int)cl.block_rank();
  const int nl = a.nlev;
  __shared__ PlaneMap pm;
  for (int l = 0; l < nl; ++l) {
    const int P = a.L[l].P;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
      int c = 0;
      while (c + 1 < kClusterCTAs && plane0(P, c + 1) <= k) ++c;
      pm.own[l][k] = (unsigned char)c;
      pm.loc[l][k] = (unsigned char)(k - plane0(P, c));
    }
  }
  {  // b of the first fused level: this block's planes
    const KLv& L = a.L[0];
    const int p0 = plane0(L.P, me), np = plane0(L.P, me + 1) - p0;
    for (int q = threadIdx.x; q < np * L.pl; q += blockDim.x) sm[L.ob + q] = a.b_in[p0 * L.pl + q];
  }
  cl.sync();
  for (int l = 0; l < nl - 1; ++l) {
    kc_smooth_pre(sm, pm, l, a.L[l], me);
    cl.sync();
    kc_residual(sm, pm, l, a.L[l], me);
    cl.sync();
    kc_restrict(sm, pm, l, a.L[l], a.L[l + 1], me);
    cl.sync();
  }
  {
    const KLv& C = a.L[nl - 1];
    if (a.dense) {
      // every block copies the whole coarsest b, then forms the rows it owns
      float* cb = sm + a.ocb;
      for (int col = threadIdx.x; col < a.nuc; col += blockDim.x) {
        const int kc = fdiv(col, C.dpl);
        cb[col] = plane_ptr(sm, pm, nl - 1, C, C.ob, kc, me)[col - kc * C.pl];
      }
      __syncthreads();
      const int p0 = plane0(C.P, me), np = plane0(C.P, me + 1) - p0;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int rr = warp; rr < np * C.pl; rr += nw) {
        const int row = p0 * C.pl + rr;
        float t = 0.f;
        for (int col = lane; col < a.nuc; col += 32) t += a.Ainv[(long long)row * a.nuc + col] * cb[col];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) sm[C.oe + rr] = t;
      }
      cl.sync();
    } else {
      kc_smooth_pre(sm, pm, nl - 1, C, me);
      cl.sync();
      for (int it = 0; it < a.coarse_sweeps; ++it) {
        kc_smooth(sm, pm, nl - 1, C, me, 1);
        cl.sync();
        kc_smooth(sm, pm, nl - 1, C, me, 0);
        cl.sync();
        kc_smooth(sm, pm, nl - 1, C, me, 0);
        cl.sync();
        kc_smooth(sm, pm, nl - 1, C, me, 1);
        cl.sync();
      }
      kc_smooth(sm, pm, nl - 1, C, me, 1);
      cl.sync();
      kc_smooth(sm, pm, nl - 1, C, me, 0);
      cl.sync();
    }
  }
  for (int l = nl - 2; l >= 0; --l) {
    kc_prolong(sm, pm, l, a.L[l], a.L[l + 1], me);
    cl.sync();
    kc_smooth(sm, pm, l, a.L[l], me, 1);
    cl.sync();
    kc_smooth(sm, pm, l, a.L[l], me, 0);
    cl.sync();
  }
  {
    const KLv& L = a.L[0];
    const int p0 = plane0(L.P, me), np = plane0(L.P, me + 1) - p0;
    for (int q = threadIdx.x; q < np * L.pl; q += blockDim.x) a.e_out[p0 * L.pl + q] = sm[L.oe + q];
  }
  cl.sync();  // no block leaves while another may still read its shared memory
}

template <class K>
struct ClusterLaunch {
  K k;
  size_t smem;
  cudaStream_t s;
  template <class... A>
  void operator()(A&&... a) const {
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClusterCTAs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCTAs);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = g_pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(a)...);
  }
};

// ---------------------------------------------------------------------------
// Exact coarse-grid solve by fast diagonalization (FP32). The level operator
// 6 e - (sum of the six neighbours) with periodic x, y and zero Dirichlet
// planes beyond the first and last unknown planes is the Kronecker sum
// C_x + C_y + T_z of two periodic second-difference matrices and one Dirichlet
// one, each diagonalized by a real orthonormal basis: Fourier cosines and sines
// in x and y, sines in z. So A^-1 b = Q (Q^T b / (lx_p + ly_q + lz_r)), Q the
// tensor product of the three bases, applied as small dense products along one
// axis at a time: per unknown plane along x and y (k_spec_plane), per column
// along z with the eigenvalue division between the two z products (k_spec_z).
// ---------------------------------------------------------------------------
struct SpecLv {
  int nx, ny, P, Pp, pl;    // cells x, y; unknown planes (Pp: padded to a multiple of 4); plane size
  // bases as columns, rows padded to 4 more floats than they hold (the shared-memory layout):
  const float* qx;          // [nx][nx + 4]: qx[i][m], basis vector m at point i
  const float* qxT;         // its transpose
  const float* qy;          // [ny][ny + 4]
  const float* qyT;
  const float* qz;          // [Pp][Pp + 4] (zero beyond P)
  const float* qzT;
  const float* lx;          // [nx] eigenvalues
  const float* ly;          // [ny]
  const float* lz;          // [Pp] (1 beyond P)
  int* timeout;             // set when a copy did not arrive in time (the solve then stops converging)
};
constexpr unsigned long long kSpecWaitNs = 1000000000ull;  // bound of every copy wait
constexpr long long kSpecMaxUnknowns = 70000;  // largest level solved this way (32 x 32 x 63 unknowns and below)

// Every thread waits for the phase; the block decides together (a wait that ran
// out anywhere marks the timeout, lets the copies in flight land, and every
// thread then leaves).
__device__ __forceinline__ bool spec_wait(uint64_t* bar, uint32_t parity, int* timeout) {
  const int late = tc::mbar_wait(bar, parity, kSpecWaitNs) ? 0 : 1;
  if (__syncthreads_or(late)) {
    if (threadIdx.x == 0 && timeout) atomicExch(timeout, 1);
    tc::mbar_wait(bar, parity, kSpecWaitNs);
    return false;
  }
  return true;
}

// C[M][N] = A[M][K] B[K][N] in shared memory, M and N multiples of 4, each
// thread a 4x4 register tile (one float4 of B and four scalars of A per step).
// Every leading dimension is a multiple of 4 and 4 more than the row it holds,
// so the four A scalars of a step (rows 4 apart) fall in different banks.
__device__ __forceinline__ void smem_gemm4(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M,
                                           int N, int K) {
  const int tn = N >> 2, tiles = (M >> 2) * tn;
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
    const int m0 = (t / tn) << 2, n0 = (t % tn) << 2;
    float acc[4][4] = {};
    for (int k = 0; k < K; ++k) {
      const float4 b = *reinterpret_cast<const float4*>(B + k * ldb + n0);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float a = A[(m0 + r) * lda + k];
        acc[r][0] = fmaf(a, b.x, acc[r][0]);
        acc[r][1] = fmaf(a, b.y, acc[r][1]);
        acc[r][2] = fmaf(a, b.z, acc[r][2]);
        acc[r][3] = fmaf(a, b.w, acc[r][3]);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      *reinterpret_cast<float4*>(C + (m0 + r) * ldc + n0) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
  }
}

// one unknown plane per block: FWD out = Qy^T (in Qx), INV out = Qy (in Qx^T);
// in and out may be the same array (a block reads its whole plane first). The
// bases and the plane's rows arrive by bulk copies on one mbarrier.
template <bool FWD>
__global__ void __launch_bounds__(256) k_spec_plane(SpecLv S, const float* in, float* out) {
  pdl_enter();
  extern __shared__ __align__(16) float sms[];
  __shared__ __align__(8) uint64_t bar;
  const int lx = S.nx + 4, ly = S.ny + 4;
  float* qx = sms;                // [nx][nx + 4]
  float* qy = qx + S.nx * lx;     // [ny][ny + 4]
  float* a = qy + S.ny * ly;      // the plane, [ny][nx + 4]
  float* t = a + S.ny * lx;       // after the x products
  const long long base = (long long)blockIdx.x * S.pl;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
    const uint32_t bx = (uint32_t)(sizeof(float) * S.nx * lx), by = (uint32_t)(sizeof(float) * S.ny * ly);
    const uint32_t row = (uint32_t)(sizeof(float) * S.nx);
    tc::mbar_arrive_expect_tx(&bar, bx + by + row * S.ny);
    tc::bulk_g2s(qx, FWD ? S.qx : S.qxT, bx, &bar);
    tc::bulk_g2s(qy, FWD ? S.qyT : S.qy, by, &bar);
    for (int j = 0; j < S.ny; ++j) tc::bulk_g2s(a + j * lx, in + base + (long long)j * S.nx, row, &bar);
  }
  __syncthreads();
  if (!spec_wait(&bar, 0, S.timeout)) return;
  smem_gemm4(a, lx, qx, lx, t, lx, S.ny, S.nx, S.nx);  // along x
  __syncthreads();
  smem_gemm4(qy, ly, t, lx, a, lx, S.ny, S.nx, S.ny);  // along y
  __syncthreads();
  const int c4 = S.nx >> 2, l4 = lx >> 2;
  for (int u = threadIdx.x; u < (S.pl >> 2); u += blockDim.x) {
    const int r = u / c4;
    reinterpret_cast<float4*>(out + base)[u] = reinterpret_cast<const float4*>(a)[r * l4 + (u - r * c4)];
  }
}

// 32 columns (x, y points) per block along z: hat = Qz^T c, hat /= eigenvalue
// sum, c = Qz hat (in place). Both bases and the columns' rows arrive by bulk
// copies on one mbarrier.
__global__ void __launch_bounds__(256) k_spec_z(SpecLv S, float* __restrict__ c) {
  pdl_enter();
  extern __shared__ __align__(16) float sms[];
  __shared__ __align__(8) uint64_t bar;
  const int Pp = S.Pp, lq = Pp + 4, lc = 36;
  float* qT = sms;            // [Pp][Pp + 4]
  float* q = qT + Pp * lq;    // [Pp][Pp + 4]
  float* a = q + Pp * lq;     // [Pp][36]
  float* h = a + Pp * lc;     // [Pp][36]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int col0 = blockIdx.x * 32, col = col0 + lane;
  const uint32_t bq = (uint32_t)(sizeof(float) * Pp * lq);
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
    tc::mbar_arrive_expect_tx(&bar, 2 * bq + (uint32_t)(128 * S.P));
    tc::bulk_g2s(qT, S.qzT, bq, &bar);
    tc::bulk_g2s(q, S.qz, bq, &bar);
    for (int k = 0; k < S.P; ++k) tc::bulk_g2s(a + k * lc, c + (long long)k * S.pl + col0, 128, &bar);
  }
  for (int k = S.P + w; k < Pp; k += nw) a[k * lc + lane] = 0.f;  // padding rows (no copy writes them)
  __syncthreads();
  if (!spec_wait(&bar, 0, S.timeout)) return;
  smem_gemm4(qT, lq, a, lc, h, lc, Pp, 32, Pp);
  __syncthreads();
  {
    const int jj = col / S.nx;
    const float lxy = S.lx[col - jj * S.nx] + S.ly[jj];
    for (int r = w; r < Pp; r += nw) h[r * lc + lane] /= lxy + S.lz[r];
  }
  __syncthreads();
  smem_gemm4(q, lq, h, lc, a, lc, Pp, 32, Pp);
  __syncthreads();
  for (int k = w; k < S.P; k += nw) c[(long long)k * S.pl + col] = a[k * lc + lane];
}

// Orthonormal eigenbasis of the periodic second difference on n points
// (columns of q, row-major [i][m]) and its eigenvalues: the constant, cosine
// and sine pairs, and for even n the alternating vector.
static void periodic_basis(int n, std::vector<double>& q, std::vector<double>& lam) {
  q.assign((size_t)n * n, 0.0);
  lam.assign(n, 0.0);
  int m = 0;
  for (int i = 0; i < n; ++i) q[(size_t)i * n + m] = 1.0 / std::sqrt((double)n);
  lam[m++] = 0.0;
  for (int f = 1; 2 * f < n; ++f) {
    const double th = 2.0 * kPi * f / n, l = 2.0 - 2.0 * std::cos(th);
    for (int i = 0; i < n; ++i) {
      q[(size_t)i * n + m] = std::sqrt(2.0 / n) * std::cos(th * i);
      q[(size_t)i * n + m + 1] = std::sqrt(2.0 / n) * std::sin(th * i);
    }
    lam[m] = lam[m + 1] = l;
    m += 2;
  }
  if (n % 2 == 0) {
    for (int i = 0; i < n; ++i) q[(size_t)i * n + m] = (i % 2 ? -1.0 : 1.0) / std::sqrt((double)n);
    lam[m++] = 4.0;
  }
}

// Dirichlet second difference on P points (zero beyond both ends): sines
static void dirichlet_basis(int P, std::vector<double>& q, std::vector<double>& lam) {
  q.assign((size_t)P * P, 0.0);
  lam.assign(P, 0.0);
  for (int r = 0; r < P; ++r) {
    const double th = kPi * (r + 1) / (P + 1);
    lam[r] = 2.0 - 2.0 * std::cos(th);
    for (int k = 0; k < P; ++k) q[(size_t)k * P + r] = std::sqrt(2.0 / (P + 1)) * std::sin(th * (k + 1));
  }
}

// largest |Q^T Q - I| entry (the bases are orthonormal to rounding)
static double ortho_err(const std::vector<double>& q, int n) {
  double e = 0.0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double d = 0.0;
      for (int i = 0; i < n; ++i) d += q[(size_t)i * n + a] * q[(size_t)i * n + b];
      e = std::max(e, std::fabs(d - (a == b ? 1.0 : 0.0)));
    }
  return e;
}

template <class T>
cudaError_t Mg<T>::init(const std::vector<MgLevel>& plan) {
  levels = plan;
  rb_ok = (plan[0].nx % 2 == 0) && (plan[0].ny % 2 == 0);
  split0 = std::is_same<T, float>::value && rb_ok && plan.size() >= 2;
  const size_t nl = plan.size();
  e.assign(nl, nullptr);
  b.assign(nl, nullptr);
  r.assign(nl, nullptr);
  cudaError_t err = cudaSuccess;
  for (size_t l = 0; l < nl; ++l) {
    const size_t bytes = sizeof(T) * (size_t)(plan[l].nu > 0 ? plan[l].nu : 1);
    if (l > 0) {
      if ((err = dev_malloc(&e[l], bytes))) return err;
      if ((err = dev_malloc(&b[l], bytes))) return err;
    }
    if ((err = dev_malloc(&r[l], bytes))) return err;
  }
  const MgLevel& c = plan.back();
  coarse_dense = rb_ok && c.nu <= 1024 && nl >= 1;
  if (coarse_dense) {
    std::vector<double> inv = dense_inverse(c);
    std::vector<T> invT(inv.begin(), inv.end());
    if ((err = dev_malloc(&Ainv, sizeof(T) * invT.size()))) return err;
    if ((err = cudaMemcpy(Ainv, invT.data(), sizeof(T) * invT.size(), cudaMemcpyHostToDevice))) return err;
  }
  // FP32: the coarse-grid correction is an exact fast-diagonalization solve at
  // the first level below the finest that allows it
  fuse_from = -1;
  fuse_smem = 0;
  spectral_at = -1;
  if constexpr (std::is_same<T, float>::value) {
    for (int l = 1; l < (int)plan.size() && rb_ok; ++l) {
      const MgLevel& M = plan[l];
      const int P = M.nz - 1;
      // the transforms cost nu (nx + ny + P) products: deep enough that this
      // stays below the per-level kernels it replaces
      if (M.nu > kSpecMaxUnknowns || M.nx > 64 || M.ny > 64 || M.nx % 4 || M.ny % 4 || (M.nx * M.ny) % 32 || P < 1 ||
          P > 128)
        continue;
      std::vector<double> qx, lx, qy, ly, qz, lz;
      periodic_basis(M.nx, qx, lx);
      periodic_basis(M.ny, qy, ly);
      dirichlet_basis(P, qz, lz);
      if (ortho_err(qx, M.nx) > 1e-10 || ortho_err(qy, M.ny) > 1e-10 || ortho_err(qz, P) > 1e-10) break;
      const int Pp = (P + 3) & ~3;
      // rows padded to 4 more floats (the kernels' shared-memory layout, one bulk copy each)
      const int lxp = M.nx + 4, lyp = M.ny + 4, lzp = Pp + 4;
      const size_t nxx = (size_t)M.nx * lxp, nyy = (size_t)M.ny * lyp, npp = (size_t)Pp * lzp;
      std::vector<float> h(2 * nxx + 2 * nyy + 2 * npp + M.nx + M.ny + Pp + 4, 0.f);
      float* hx = h.data();
      float* hxT = hx + nxx;
      float* hy = hxT + nxx;
      float* hyT = hy + nyy;
      float* hz = hyT + nyy;
      float* hzT = hz + npp;
      float* hlx = hzT + npp;
      float* hly = hlx + M.nx;
      float* hlz = hly + M.ny;
      for (int i = 0; i < M.nx; ++i)
        for (int m = 0; m < M.nx; ++m) {
          hx[(size_t)i * lxp + m] = (float)qx[(size_t)i * M.nx + m];
          hxT[(size_t)m * lxp + i] = (float)qx[(size_t)i * M.nx + m];
        }
      for (int j = 0; j < M.ny; ++j)
        for (int m = 0; m < M.ny; ++m) {
          hy[(size_t)j * lyp + m] = (float)qy[(size_t)j * M.ny + m];
          hyT[(size_t)m * lyp + j] = (float)qy[(size_t)j * M.ny + m];
        }
      for (int k = 0; k < P; ++k)
        for (int r = 0; r < P; ++r) {
          hz[(size_t)k * lzp + r] = (float)qz[(size_t)k * P + r];
          hzT[(size_t)r * lzp + k] = (float)qz[(size_t)k * P + r];
        }
      for (int i = 0; i < M.nx; ++i) hlx[i] = (float)lx[i];
      for (int j = 0; j < M.ny; ++j) hly[j] = (float)ly[j];
      for (int r = 0; r < Pp; ++r) hlz[r] = r < P ? (float)lz[r] : 1.f;
      if ((err = dev_malloc(&spec_mem, sizeof(float) * h.size()))) return err;
      if ((err = cudaMemcpy(spec_mem, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice))) return err;
      spec_smem_plane = sizeof(float) * (nxx + nyy + 2 * (size_t)M.ny * lxp);
      spec_smem_z = sizeof(float) * (2 * npp + 72 * (size_t)Pp);
      // the attribute is the kernel's, shared by every solver of the process:
      // set to what the largest admitted level needs (64 x 64, 128 planes)
      const int plane_max = (int)sizeof(float) * (4 * 64 * 68);
      const int z_max = (int)sizeof(float) * (2 * 128 * 132 + 72 * 128);
      bool ok = cudaFuncSetAttribute(k_spec_plane<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, plane_max) ==
                    cudaSuccess &&
                cudaFuncSetAttribute(k_spec_plane<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, plane_max) ==
                    cudaSuccess &&
                cudaFuncSetAttribute(k_spec_z, cudaFuncAttributeMaxDynamicSharedMemorySize, z_max) == cudaSuccess;
      cudaGetLastError();
      if (ok) spectral_at = l;
      break;
    }
  }
  // FP32 without that solve: the deepest levels whose e, b, r fit in the shared
  // memory of a cluster's blocks run in k_coarse_cluster (at least two levels,
  // never level 0)
  if constexpr (std::is_same<T, float>::value) {
    if (spectral_at > 0) return cudaSuccess;
    const size_t cap = 200 * 1024;
    const int nl_ = (int)plan.size();
    int best = -1;
    size_t floats = 0, best_floats = 0;
    for (int l = nl_ - 1; l >= 1; --l) {
      const long long P = plan[l].nz - 1, pl = (long long)plan[l].nx * plan[l].ny;
      const long long maxp = (P + kClusterCTAs - 1) / kClusterCTAs;
      floats += (size_t)(3 * maxp * pl);
      const size_t extra = coarse_dense ? (size_t)plan[nl_ - 1].nu : 0;  // local copy of the coarsest b
      // the cluster's 8 SMs issue every phase: levels above ~16 K unknowns are
      // faster as grid-wide kernels on all SMs
      if (sizeof(float) * (floats + extra) > cap || nl_ - l > kMaxFused || P > kMaxPlanes ||
          plan[l].nu > kClusterMaxUnknowns)
        break;
      if (nl_ - l >= 2) {
        best = l;
        best_floats = floats + extra;
      }
    }
    if (rb_ok && best > 0) {
      const size_t bytes = sizeof(float) * best_floats;
      // the attribute is the kernel's, shared by every solver of the process: the
      // cap of the selection above, so that every instance's launch fits
      bool ok = cudaFuncSetAttribute(k_coarse_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap) ==
                cudaSuccess;
      if (ok) {  // can a cluster of this size be resident at all?
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kClusterCTAs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kClusterCTAs);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.dynamicSmemBytes = bytes;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        ok = cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_cluster, &cfg) == cudaSuccess && nclusters > 0;
      }
      cudaGetLastError();
      if (ok) {
        fuse_from = best;
        fuse_smem = bytes;
      }
    }
  }
  return cudaSuccess;
}

template <class T>
void Mg<T>::release() {
  for (auto* p : e) dev_free(p);
  for (auto* p : b) dev_free(p);
  for (auto* p : r) dev_free(p);
  e.clear();
  b.clear();
  r.clear();
  if (Ainv) dev_free(Ainv);
  Ainv = nullptr;
  if (spec_mem) dev_free(spec_mem);
  spec_mem = nullptr;
  spectral_at = -1;
}

// z = M^-1 rhs (one V(1,1) cycle from zero); rhs and z live at level 0 outside
template <class T>
bool Mg<T>::vcycle(const T* rhs, T* z, cudaStream_t s, double* part, SolveCtl* ctl) {
  const int nl = (int)levels.size();
  bool dot_done = false;
  if (!rb_ok) {
    // Jacobi preconditioner: z = rhs / 6
    const Lv L = lv_of(levels[0]);
    SOLVER_LAUNCH(sgrid(L.nu), kSB, 0, s, k_copy<T>)(L.nu, z, rhs);
    SOLVER_LAUNCH(sgrid(L.nu), kSB, 0, s, k_jacobi_scale<T>)(L.nu, z);
    return false;
  }
  std::vector<T*> E(nl), B(nl);
  for (int l = 0; l < nl; ++l) {
    E[l] = l == 0 ? z : e[l];
    B[l] = l == 0 ? const_cast<T*>(rhs) : b[l];
  }
  const int ff = fuse_from;  // levels ff..nl-1 run in one cluster (FP32 only), -1: none
  const int sp = spectral_at;  // level solved exactly (FP32 only), -1: none
  const int bottom = sp > 0 ? sp : (ff > 0 ? ff : nl - 1);
  for (int l = 0; l < bottom; ++l) {
    const Lv L = lv_of(levels[l]);
    const Lv C = lv_of(levels[l + 1]);
    if (l == 0 && split0) {
      SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_smooth_pre_s<T>)(L, E[l], B[l]);
      SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_residual_s<T>)(L, E[l], B[l], r[l]);
      SOLVER_LAUNCH(g3(C, C.nx), kB3, 0, s, k_restrict_s0<T>)(L, C, r[l], B[l + 1]);
      continue;
    }
    SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_smooth_pre<T>)(L, E[l], B[l]);
    SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_residual<T>)(L, E[l], B[l], r[l]);
    SOLVER_LAUNCH(g3(C, C.nx), kB3, 0, s, k_restrict<T>)(L, C, r[l], B[l + 1]);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (sp > 0) {
      const MgLevel& M = levels[sp];
      SpecLv S;
      S.nx = M.nx;
      S.ny = M.ny;
      S.P = M.nz - 1;
      S.Pp = (S.P + 3) & ~3;
      S.pl = M.nx * M.ny;
      const size_t nxx = (size_t)M.nx * (M.nx + 4), nyy = (size_t)M.ny * (M.ny + 4), npp = (size_t)S.Pp * (S.Pp + 4);
      S.timeout = ctl ? &ctl->spec_timeout : nullptr;
      S.qx = spec_mem;
      S.qxT = S.qx + nxx;
      S.qy = S.qxT + nxx;
      S.qyT = S.qy + nyy;
      S.qz = S.qyT + nyy;
      S.qzT = S.qz + npp;
      S.lx = S.qzT + npp;
      S.ly = S.lx + M.nx;
      S.lz = S.ly + M.ny;
      // e = A^-1 b at this level: forward transforms into e, per-column solve, inverse transforms
      SOLVER_LAUNCH(S.P, 256, spec_smem_plane, s, k_spec_plane<true>)(S, B[sp], E[sp]);
      SOLVER_LAUNCH((S.pl + 31) / 32, 256, spec_smem_z, s, k_spec_z)(S, E[sp]);
      SOLVER_LAUNCH(S.P, 256, spec_smem_plane, s, k_spec_plane<false>)(S, E[sp], E[sp]);
    }
    if (sp <= 0 && ff > 0) {
      ClusterArgs ca{};
      ca.nlev = nl - ff;
      int off = 0;
      for (int q = 0; q < ca.nlev; ++q) {
        const MgLevel& M = levels[ff + q];
        KLv& c = ca.L[q];
        c.nx = M.nx;
        c.ny = M.ny;
        c.P = M.nz - 1;
        c.pl = M.nx * M.ny;
        c.hx = M.nx / 2;
        c.dnx = make_fastdiv(c.nx);
        c.dpl = make_fastdiv(c.pl);
        c.dhx = make_fastdiv(c.hx);
        c.dhxny = make_fastdiv(c.hx * c.ny);
        c.maxp = (c.P + kClusterCTAs - 1) / kClusterCTAs;
        c.oe = off;
        c.ob = off + c.maxp * c.pl;
        c.orr = off + 2 * c.maxp * c.pl;
        off += 3 * c.maxp * c.pl;
      }
      ca.dense = coarse_dense ? 1 : 0;
      ca.nuc = (int)levels[nl - 1].nu;
      ca.ocb = off;
      ca.coarse_sweeps = coarse_sweeps;
      ca.Ainv = Ainv;
      ca.b_in = B[ff];
      ca.e_out = E[ff];
      count_kernel();
      ClusterLaunch<decltype(&k_coarse_cluster)>{&k_coarse_cluster, fuse_smem, s}(ca);
    }
  }
  if (sp <= 0 && ff <= 0) {
    const Lv C = lv_of(levels[nl - 1]);
    if (coarse_dense) {
      const int cg = (int)std::min<long long>((C.nu * 32 + kSB - 1) / kSB, 4096);
      SOLVER_LAUNCH(cg, kSB, 0, s, k_coarse<T>)(C.nu, Ainv, B[nl - 1],
                                                                                              E[nl - 1]);
    } else {
      SOLVER_LAUNCH(g3(C, C.nx / 2), kB3, 0, s, k_smooth_pre<T>)(C, E[nl - 1], B[nl - 1]);
      for (int it = 0; it < coarse_sweeps; ++it) {
        SOLVER_LAUNCH(g3(C, C.nx / 2), kB3, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 1);
        SOLVER_LAUNCH(g3(C, C.nx / 2), kB3, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 0);
        SOLVER_LAUNCH(g3(C, C.nx / 2), kB3, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 0);
        SOLVER_LAUNCH(g3(C, C.nx / 2), kB3, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 1);
      }
      SOLVER_LAUNCH(g3(C, C.nx / 2), kB3, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 1);
      SOLVER_LAUNCH(g3(C, C.nx / 2), kB3, 0, s, k_smooth<T>)(C, E[nl - 1], B[nl - 1], 0);
    }
  }
  for (int l = bottom - 1; l >= 0; --l) {
    const Lv L = lv_of(levels[l]);
    const Lv C = lv_of(levels[l + 1]);
    if (l == 0 && split0) {
      SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_prolong_s0<T>)(L, C, E[l + 1], E[l]);
      SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_smooth_s<T>)(L, E[l], B[l], 1);
      if (ctl) {
        SOLVER_LAUNCH(g3rs(L), kB3, 0, s, k_smooth_s_dot<T>)(L, E[l], B[l], part, ctl);
        dot_done = true;
      } else {
        SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_smooth_s<T>)(L, E[l], B[l], 0);
      }
      continue;
    }
    SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_prolong<T>)(L, C, E[l + 1], E[l]);
    SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_smooth<T>)(L, E[l], B[l], 1);
    SOLVER_LAUNCH(g3(L, L.nx / 2), kB3, 0, s, k_smooth<T>)(L, E[l], B[l], 0);
  }
  return dot_done;
}

// ---------------------------------------------------------------------------
// Device-controlled solve. All scalars live in SolveCtl on the device; the
// stopping decisions set the conditional handles of two nested WHILE nodes of a
// CUDA graph (outer: FP64 true residual / refinement; inner: PCG iterations),
// so a solve is one graph launch with no host round trip.
// ---------------------------------------------------------------------------
template <class V>
__device__ __forceinline__ V warp_sum(V d) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  return d;
}

// Grid-wide sum without a second launch: each block stores its partial in
// part[block], then the last block to arrive (a ticket counter) adds all
// partials in a fixed order (fixed thread assignment and tree, so the total is
// reproducible) and resets the ticket. Returns true in thread 0 of that block
// only, with the total in *tot. Every thread of every block must call it.
// Per-thread and warp sums stay in V (FP32 for the FP32 solve: FP64 is a narrow
// pipe on GB300); warp totals and everything above them are FP64.
template <class V>
__device__ __forceinline__ bool grid_total(V v, double* part, unsigned* ticket, double* tot) {
  __shared__ double sm[32];
  __shared__ int s_last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  const int nw = nthr >> 5;
  const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
  const V w = warp_sum(v);
  if ((tid & 31) == 0) sm[tid >> 5] = (double)w;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sm[k];
    part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == nb - 1u ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  // four independent partial sums per thread keep several loads in flight
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  unsigned i = tid;
  for (; i + 3u * nthr < nb; i += 4u * nthr) {
    s0 += __ldcg(part + i);
    s1 += __ldcg(part + i + nthr);
    s2 += __ldcg(part + i + 2u * nthr);
    s3 += __ldcg(part + i + 3u * nthr);
  }
  for (; i < nb; i += nthr) s0 += __ldcg(part + i);
  double s = warp_sum((s0 + s1) + (s2 + s3));
  __syncthreads();
  if ((tid & 31) == 0) sm[tid >> 5] = s;
  __syncthreads();
  if (tid != 0) return false;
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += sm[k];
  *tot = t;
  *ticket = 0u;
  return true;
}

__device__ __forceinline__ void fin_bb(double bb, SolveCtl* c, double rtol, int maxit) {
  c->bb = bb;
  c->tol2 = rtol * rtol * bb;
  c->it_total = 0;
  c->outer = 0;
  c->converged = bb == 0.0 ? 1 : 0;
  c->maxit = maxit;
  c->rr_true = 0.0;
  c->resid_rel = 0.0;
}

// b.b -> tolerance; start of a solve
__global__ void __launch_bounds__(kSB) k_dot_bb(int n, const double* __restrict__ b, double* part, SolveCtl* c,
                                                double rtol, int maxit) {
  pdl_enter();
  double acc = 0.0;
  for (int u = blockIdx.x * kSB + threadIdx.x; u < n; u += gridDim.x * kSB) acc += b[u] * b[u];
  double bb;
  if (grid_total(acc, part, &c->ticket, &bb)) fin_bb(bb, c, rtol, maxit);
}

// The mixed path's inner (FP32) solve stops once its recursive residual is
// below 0.9 of the outer tolerance (kInnerMargin2 = 0.9^2 on r.r): the
// float-float residual the outer loop then takes differs from it only by the
// FP32 rounding of the correction, about 1e-7 of the residual the inner solve
// started from, far inside the margin.
constexpr double kInnerMargin2 = 0.81;

// Outer-loop decision from the true residual r.r (last block of a residual kernel)
__device__ __forceinline__ void fin_outer(double rr, SolveCtl* c, cudaGraphConditionalHandle h_outer,
                                          cudaGraphConditionalHandle h_inner, double inner_rtol, int mixed,
                                          int max_outer, int use_graph) {
  c->ax_valid = 1;
  c->rr_true = rr;
  c->resid_rel = c->bb > 0.0 ? sqrt(rr / c->bb) : 0.0;
  const bool done = c->bb == 0.0 || rr <= c->tol2 || !(rr == rr) || c->it_total >= c->maxit || c->outer >= max_outer;
  c->converged = (c->bb == 0.0 || rr <= c->tol2) ? 1 : 0;
  c->rr = rr;
  c->it_inner = 0;
  c->tol_in2 = mixed ? fmax(inner_rtol * inner_rtol * rr, kInnerMargin2 * c->tol2) : c->tol2;
  c->outer += 1;
  c->more = done ? 0 : 1;
  c->stopped = done ? 1 : 0;
  if (use_graph) {
    cudaGraphSetConditional(h_outer, done ? 0u : 1u);
    cudaGraphSetConditional(h_inner, done ? 0u : 1u);
  }
}

// r_in = (Tin)(b - A x) with x, b FP64 (x = 0 when b = 0); d = 0; then, in the last block, the
// outer-loop decision from r.r (FP64). A x is kept in ax: while c->ax_valid is
// set, ax holds A x for the current x (x unchanged since it was written), and
// the residual is b - ax without the stencil.
template <class Tin>
__global__ void __launch_bounds__(256) k_residual_prep(Lv L, double* __restrict__ x, const double* __restrict__ b,
                                                       double* __restrict__ ax, Tin* __restrict__ r_in,
                                                       Tin* __restrict__ d, double* part, SolveCtl* c,
                                                       cudaGraphConditionalHandle h_outer,
                                                       cudaGraphConditionalHandle h_inner, double inner_rtol,
                                                       int mixed, int max_outer, int use_graph) {
  pdl_enter();
  Tin acc = 0;
  const bool zero_x = c->bb == 0.0;
  const bool cached = c->ax_valid != 0;
  ROWS3K(L, L.nx) {
    if (!in_x) continue;
    const int u = k * L.pl + j * L.nx + i;
    double rv = 0.0;
    if (zero_x) {  // b = 0: the solution is x = 0
      x[u] = 0.0;
      ax[u] = 0.0;
    } else {
      double axv;
      if (cached) {
        axv = ax[u];
      } else {
        axv = 6.0 * x[u] - nb_sum(L, x, u, i, j, k);
        ax[u] = axv;
      }
      rv = b[u] - axv;
    }
    const Tin ri = (Tin)rv;
    r_in[u] = ri;
    d[u] = (Tin)0;
    acc += ri * ri;
  }
  double rr;
  if (grid_total(acc, part, &c->ticket, &rr))
    fin_outer(rr, c, h_outer, h_inner, inner_rtol, mixed, max_outer, use_graph);
}

// ---------------------------------------------------------------------------
// MIXED path: the outer loop in float-float arithmetic. Over the unknowns the
// potential is kept as phi = vac(k) + hi + lo, with hi and lo FP32 and hi the
// FP32 deviation from the vacuum potential vac(k) = phi_c + k (phi_a - phi_c)/nz
// that the field kernel reads (phi32). The linear vac satisfies A vac = the
// folded Dirichlet terms, so b - A phi = f - A (hi + lo), f = fl32(h^2 rho/eps0)
// the FP32 charge term. A hi is summed with error-free transformations (Knuth's
// TwoSum; 6 hi exactly as a product and its FMA remainder), A lo in plain FP32:
// the residual carries about 48 significant bits with no FP64 instruction (FP64
// is a narrow pipe on GB300). The _rn intrinsics keep the compiler from fusing
// the products and sums the transformations rely on.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// sum of the six neighbours of u as s + e (s rounded, e the accumulated exact errors)
__device__ __forceinline__ void nb_sum_ff(const Lv& L, const float* __restrict__ x, int u, int i, int j, int k, float& s,
                                          float& e) {
  const int row = u - i;
  const int im = i == 0 ? L.nx - 1 : i - 1, ip = i == L.nx - 1 ? 0 : i + 1;
  const int rm = j == 0 ? (L.ny - 1) * L.nx : -L.nx;
  const int rp = j == L.ny - 1 ? -(L.ny - 1) * L.nx : L.nx;
  float t;
  s = x[row + im];
  e = 0.f;
  two_sum(s, x[row + ip], s, t);
  e = __fadd_rn(e, t);
  two_sum(s, x[u + rm], s, t);
  e = __fadd_rn(e, t);
  two_sum(s, x[u + rp], s, t);
  e = __fadd_rn(e, t);
  if (k > 0) {
    two_sum(s, x[u - L.pl], s, t);
    e = __fadd_rn(e, t);
  }
  if (k < L.nz - 2) {
    two_sum(s, x[u + L.pl], s, t);
    e = __fadd_rn(e, t);
  }
}

// sum f.f + folded terms -> tolerance (b = f + fold never materialised). f is
// natural ([k][j][i], planes of nx ny) over the unknown planes, so this is a
// flat pass: four values per thread (16-byte loads) where the plane size keeps
// the planes 16-byte aligned (a float4 then never straddles two planes).
__global__ void __launch_bounds__(kSB) k_dot_bb_ff(Lv L, const float* __restrict__ f, float fold_first, float fold_last,
                                                   double* part, SolveCtl* c, double rtol, int maxit) {
  pdl_enter();
  const long long pl = L.pl;
  const long long nu = (long long)(L.nz - 1) * pl;
  const long long last = nu - pl;  // first unknown of the plane next to the anode
  auto sq = [&](float bv, long long u) -> float {
    if (u < pl) bv += fold_first;
    if (u >= last) bv += fold_last;
    return bv * bv;
  };
  float acc = 0.f;
  long long u0 = 0;
  if ((pl & 3) == 0) {
    const float4* f4 = reinterpret_cast<const float4*>(f);
    const long long n4 = nu >> 2;
    for (long long q = gtid(); q < n4; q += gstride()) {
      const float4 v = f4[q];
      const long long u = q << 2;
      acc += (sq(v.x, u) + sq(v.y, u)) + (sq(v.z, u) + sq(v.w, u));
    }
    u0 = n4 << 2;
  }
  for (long long u = u0 + gtid(); u < nu; u += gstride()) acc += sq(f[u], u);
  double bb;
  if (grid_total(acc, part, &c->ticket, &bb)) fin_bb(bb, c, rtol, maxit);
}

// r = fl32(f - A (hi + lo)); d = 0; outer decision in the last block.
// b = 0 (bb = 0): the solution is phi = 0, i.e. hi + lo = -vac.
// split: r and d are in the colour-split layout of the finest level (hi, lo, f natural)
__global__ void __launch_bounds__(256) k_residual_ff(Lv L, float* __restrict__ hi, float* __restrict__ lo,
                                                     const float* __restrict__ f, float* __restrict__ r,
                                                     float* __restrict__ d, double phi_c, double dphi_dk, double* part,
                                                     SolveCtl* c, cudaGraphConditionalHandle h_outer,
                                                     cudaGraphConditionalHandle h_inner, double inner_rtol,
                                                     int max_outer, int use_graph, int split) {
  pdl_enter();
  float acc = 0.f;
  const bool zero_x = c->bb == 0.0;
  ROWS3K(L, L.nx) {
    if (!in_x) continue;
    const int u = k * L.pl + j * L.nx + i;
    float rv = 0.f;
    if (zero_x) {
      const double v = -(phi_c + dphi_dk * (double)(k + 1));
      const float vh = (float)v;
      hi[u] = vh;
      lo[u] = (float)(v - (double)vh);
    } else {
      float s, e;
      nb_sum_ff(L, hi, u, i, j, k, s, e);
      const float hc = hi[u];
      const float p6 = __fmul_rn(6.f, hc);
      const float e6 = __fmaf_rn(6.f, hc, -p6);  // 6 hc = p6 + e6 exactly
      float a1, ea;
      two_sum(p6, -s, a1, ea);  // A hi = a1 + ea + e6 - e
      const float alo = __fsub_rn(__fmul_rn(6.f, lo[u]), nb_sum(L, lo, u, i, j, k));
      float r1, er;
      two_sum(f[u], -a1, r1, er);
      const float small = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(er, ea), e6), e), alo);
      rv = __fadd_rn(r1, small);
    }
    const int w = split ? sp_index(L, i, j, k) : u;
    r[w] = rv;
    d[w] = 0.f;
    acc += rv * rv;
  }
  double rr;
  if (grid_total(acc, part, &c->ticket, &rr))
    fin_outer(rr, c, h_outer, h_inner, inner_rtol, 1, max_outer, use_graph);
}

// (hi, lo) += d, renormalised (hi = fl32(hi + lo)); nothing to do once stopped.
// split: d in the colour-split layout of the finest level.
__global__ void __launch_bounds__(256) k_update_ff(Lv L, float* __restrict__ hi, float* __restrict__ lo,
                                                   const float* __restrict__ d, const SolveCtl* c, int split) {
  pdl_enter();
  if (c->stopped) return;
  ROWS3(L, L.nx) {
    if (!in_x) continue;
    const int u = k * L.pl + j * L.nx + i;
    const float dv = d[split ? sp_index(L, i, j, k) : u];
    float s, e;
    two_sum(hi[u], dv, s, e);
    e = __fadd_rn(e, lo[u]);
    const float h2 = __fadd_rn(s, e);
    hi[u] = h2;
    lo[u] = __fsub_rn(e, __fsub_rn(h2, s));
  }
}

// phi (FP64, unknown view) = vac + hi + lo
__global__ void __launch_bounds__(256) k_phi_from_ff(Lv L, const float* __restrict__ hi, const float* __restrict__ lo,
                                                     double* __restrict__ x, double phi_c, double dphi_dk) {
  pdl_enter();
  const double vac = phi_c + dphi_dk * (double)(blockIdx.z + 1);
  ROWS3(L, L.nx) {
    if (!in_x) continue;
    const int u = k * L.pl + j * L.nx + i;
    x[u] = vac + ((double)hi[u] + (double)lo[u]);
  }
}

// (hi, lo) from phi (FP64, unknown view; nullptr: phi = 0)
__global__ void __launch_bounds__(256) k_ff_from_phi(Lv L, const double* __restrict__ x, float* __restrict__ hi,
                                                     float* __restrict__ lo, double phi_c, double dphi_dk) {
  pdl_enter();
  const double vac = phi_c + dphi_dk * (double)(blockIdx.z + 1);
  ROWS3(L, L.nx) {
    if (!in_x) continue;
    const int u = k * L.pl + j * L.nx + i;
    const double v = (x ? x[u] : 0.0) - vac;
    const float vh = (float)v;
    hi[u] = vh;
    lo[u] = (float)(v - (double)vh);
  }
}

// r.z -> beta
// The streaming PCG kernels move FP32 vectors as float4 (16-byte loads keep
// four times the bytes in flight per load); the FP64 instantiations and the
// tail after the last full float4 go element by element. The level-0 vectors
// are separate allocations, hence 16-byte aligned.
// r.z of this iteration -> beta (0 on the first iteration of an inner solve)
__device__ __forceinline__ void set_beta(SolveCtl* c, double rz) {
  c->beta = c->it_inner > 0 ? rz / c->rz : 0.0;
  c->rz = rz;
}

template <class T>
struct Vec4 {
  static constexpr bool on = false;
};
template <>
struct Vec4<float> {
  static constexpr bool on = true;
};

// r.z -> beta
template <class T>
__global__ void __launch_bounds__(kSB) k_dot_rz(int n, const T* __restrict__ r, const T* __restrict__ z, double* part,
                                                SolveCtl* c) {
  pdl_enter();
  T acc = 0;
  int u0 = 0;
  if constexpr (Vec4<T>::on) {
    const int n4 = n >> 2;
    const float4* r4 = reinterpret_cast<const float4*>(r);
    const float4* z4 = reinterpret_cast<const float4*>(z);
    for (int q = blockIdx.x * kSB + threadIdx.x; q < n4; q += gridDim.x * kSB) {
      const float4 a = r4[q], b = z4[q];
      acc += (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w);
    }
    u0 = n4 * 4;
  }
  for (int u = u0 + blockIdx.x * kSB + threadIdx.x; u < n; u += gridDim.x * kSB) acc += r[u] * z[u];
  double rz;
  if (grid_total(acc, part, &c->ticket, &rz)) set_beta(c, rz);
}

// q = A p ; p.q -> alpha
template <class T>
__global__ void __launch_bounds__(256) k_apply_pq(Lv L, const T* __restrict__ p, T* __restrict__ q, double* part,
                                                  SolveCtl* c) {
  pdl_enter();
  T acc = 0;
  ROWS3K(L, L.nx) {
    if (!in_x) continue;
    const int u = k * L.pl + j * L.nx + i;
    const T pv = p[u];
    const T qv = (T)6 * pv - nb_sum(L, p, u, i, j, k);
    q[u] = qv;
    acc += pv * qv;
  }
  double pq;
  if (!grid_total(acc, part, &c->ticket, &pq)) return;
  c->pq = pq;
  c->alpha = pq != 0.0 ? c->rz / pq : 0.0;
}

// q = A p ; p.q -> alpha, on the split finest level (both colours per thread;
// planes strided as in the natural kernel, at most one wave of blocks)
// the centre and the six neighbours of one point (absent z neighbours 0)
template <class T>
struct Pt7 {
  T c, xm, xp, ym, yp, zm, zp;
};
template <class T>
__device__ __forceinline__ Pt7<T> load_pt7(const T* __restrict__ self, const T* __restrict__ o, int at, const SpNb& n) {
  Pt7<T> v;
  v.c = self[at];
  v.xm = o[n.xm];
  v.xp = o[n.xp];
  v.ym = o[n.ym];
  v.yp = o[n.yp];
  v.zm = n.zm >= 0 ? o[n.zm] : (T)0;
  v.zp = n.zp >= 0 ? o[n.zp] : (T)0;
  return v;
}
// 6 c - the neighbours, summed in sp_sum's order (adding an absent 0 is exact)
template <class T>
__device__ __forceinline__ T apply_pt7(const Pt7<T>& v) {
  return (T)6 * v.c - (((((v.xm + v.xp) + v.ym) + v.yp) + v.zm) + v.zp);
}

template <class T>
__global__ void __launch_bounds__(256) k_apply_pq_s(Lv L, const T* __restrict__ p, T* __restrict__ q, double* part,
                                                    SolveCtl* c) {
  pdl_enter();
  T acc = 0;
  const int m = blockIdx.x * kBX + threadIdx.x;
  const int hx = L.nx >> 1, half = L.nu >> 1;
  if (m < hx) {
    // both colours of a point per pass, their fourteen loads issued together
    for (int k = blockIdx.z; k < L.nz - 1; k += gridDim.z)
      for (int j = blockIdx.y * kBY + threadIdx.y; j < L.ny; j += gridDim.y * kBY) {
        const int row = (k * L.ny + j) * hx + m;
        const SpNb n0 = sp_nb(L, m, j, k, (j + k + 1) & 1);
        const SpNb n1 = sp_nb(L, m, j, k, (j + k) & 1);
        const Pt7<T> a = load_pt7(p, p + half, row, n0);
        const Pt7<T> b = load_pt7(p + half, p, row, n1);
        const T qa = apply_pt7(a), qb = apply_pt7(b);
        q[row] = qa;
        q[half + row] = qb;
        acc += a.c * qa;
        acc += b.c * qb;
      }
  }
  double pq;
  if (!grid_total(acc, part, &c->ticket, &pq)) return;
  c->pq = pq;
  c->alpha = pq != 0.0 ? c->rz / pq : 0.0;
}

// p = z (first iteration of this inner solve) or z + beta p
template <class T>
__global__ void __launch_bounds__(kSB) k_pupdate_c(long long n, T* __restrict__ p, const T* __restrict__ z, const SolveCtl* c) {
  pdl_enter();
  const bool first = c->it_inner == 0;
  const T beta = first ? (T)0 : (T)c->beta;
  long long u0 = 0;
  if constexpr (Vec4<T>::on) {
    const long long n4 = n >> 2;
    float4* p4 = reinterpret_cast<float4*>(p);
    const float4* z4 = reinterpret_cast<const float4*>(z);
    for (long long q = gtid(); q < n4; q += gstride()) {
      const float4 zv = z4[q];
      if (first) {
        p4[q] = zv;
      } else {
        const float4 pv = p4[q];
        p4[q] = make_float4(zv.x + beta * pv.x, zv.y + beta * pv.y, zv.z + beta * pv.z, zv.w + beta * pv.w);
      }
    }
    u0 = n4 * 4;
  }
  for (long long u = u0 + gtid(); u < n; u += gstride()) p[u] = first ? z[u] : z[u] + beta * p[u];
}

// d += alpha p ; r -= alpha q ; r.r -> inner-loop decision
template <class T>
__global__ void __launch_bounds__(kSB) k_update_rr(long long n, T* __restrict__ d, T* __restrict__ r, const T* __restrict__ p,
                                                   const T* __restrict__ q, SolveCtl* c, double* part,
                                                   cudaGraphConditionalHandle h_inner, int use_graph) {
  pdl_enter();
  const T alpha = (T)c->alpha;
  T acc = 0;
  long long u0 = 0;
  if constexpr (Vec4<T>::on) {
    const long long n4 = n >> 2;
    float4* d4 = reinterpret_cast<float4*>(d);
    float4* r4 = reinterpret_cast<float4*>(r);
    const float4* p4 = reinterpret_cast<const float4*>(p);
    const float4* q4 = reinterpret_cast<const float4*>(q);
    for (long long w = gtid(); w < n4; w += gstride()) {
      const float4 pv = p4[w], qv = q4[w];
      float4 dv = d4[w], rv = r4[w];
      dv.x += alpha * pv.x;
      dv.y += alpha * pv.y;
      dv.z += alpha * pv.z;
      dv.w += alpha * pv.w;
      rv.x -= alpha * qv.x;
      rv.y -= alpha * qv.y;
      rv.z -= alpha * qv.z;
      rv.w -= alpha * qv.w;
      d4[w] = dv;
      r4[w] = rv;
      acc += (rv.x * rv.x + rv.y * rv.y) + (rv.z * rv.z + rv.w * rv.w);
    }
    u0 = n4 * 4;
  }
  for (long long u = u0 + gtid(); u < n; u += gstride()) {
    d[u] += alpha * p[u];
    const T rv = r[u] - alpha * q[u];
    r[u] = rv;
    acc += rv * rv;
  }
  double rr;
  if (!grid_total(acc, part, &c->ticket, &rr)) return;
  c->rr = rr;
  c->it_inner += 1;
  c->it_total += 1;
  const bool more = rr > c->tol_in2 && c->it_total < c->maxit && (rr == rr);
  c->more = more ? 1 : 0;
  if (use_graph) cudaGraphSetConditional(h_inner, more ? 1u : 0u);
}

// x += d (FP64); optionally phi32 = (float)(x - phi_vac(z)) on the same nodes.
// Unless the outer loop has just stopped (then d = 0 and x stays as it is), x
// changes and the kept A x is no longer valid.
template <class T>
__global__ void __launch_bounds__(256) k_axpy_out(Lv L, double* __restrict__ x, const T* __restrict__ d, float* __restrict__ phi32,
                                                  double phi_c, double dphi_dk, SolveCtl* c) {
  pdl_enter();
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0 && !c->stopped)
    c->ax_valid = 0;
  const double vac = phi_c + dphi_dk * (double)(blockIdx.z + 1);  // vacuum potential of this node plane
  ROWS3(L, L.nx) {
    if (!in_x) continue;
    const int u = k * L.pl + j * L.nx + i;
    const double v = x[u] + (double)d[u];
    x[u] = v;
    if (phi32) phi32[u] = (float)(v - vac);
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
  if ((err = dev_malloc(&r, bytes))) return err;
  if ((err = dev_malloc(&z, bytes))) return err;
  if ((err = dev_malloc(&p, bytes))) return err;
  if ((err = dev_malloc(&q, bytes))) return err;
  if ((err = dev_malloc(&d, bytes))) return err;
  if ((err = cudaMemset(p, 0, bytes))) return err;
  if ((err = cudaMemset(d, 0, bytes))) return err;
  return mg.init(plan);
}

template <class T>
void Pcg<T>::release() {
  dev_free(r);
  dev_free(z);
  dev_free(p);
  dev_free(q);
  dev_free(d);
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
  const size_t nn = (size_t)(n > 0 ? n : 1);
  if (precision == 0) {
    if ((err = dev_malloc(&b, sizeof(double) * nn))) return err;
    if ((err = cudaMemset(b, 0, sizeof(double) * nn))) return err;
    if ((err = dev_malloc(&ax, sizeof(double) * nn))) return err;
  } else {
    if ((err = dev_malloc(&f32, sizeof(float) * nn))) return err;
    if ((err = cudaMemset(f32, 0, sizeof(float) * nn))) return err;
    if ((err = dev_malloc(&lo32, sizeof(float) * nn))) return err;
    if ((err = cudaMemset(lo32, 0, sizeof(float) * nn))) return err;
  }
  if ((err = dev_malloc(&part, sizeof(double) * kPartsMax))) return err;
  if ((err = dev_malloc(&ctl, sizeof(SolveCtl)))) return err;
  if ((err = cudaMemset(ctl, 0, sizeof(SolveCtl)))) return err;
  if ((err = cudaMallocHost(&host_ctl, sizeof(SolveCtl)))) return err;
  memset(host_ctl, 0, sizeof(SolveCtl));
  for (auto& a : aux)
    if ((err = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking))) return err;
  if (precision == 0) return p64.init(plan);
  return p32.init(plan);
}

void Solver::release() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  dev_free(b);
  dev_free(ax);
  dev_free(f32);
  dev_free(lo32);
  dev_free(part);
  dev_free(ctl);
  if (host_ctl) cudaFreeHost(host_ctl);
  host_ctl = nullptr;
  for (auto& a : aux) {
    if (a) cudaStreamDestroy(a);
    a = nullptr;
  }
  b = nullptr;
  ax = nullptr;
  f32 = nullptr;
  lo32 = nullptr;
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
  if (!pc.mg.vcycle(pc.r, pc.z, s, part, ctl)) SOLVER_LAUNCH(G, kSB, 0, s, k_dot_rz<T>)(L.nu, pc.r, pc.z, part, ctl);
  const dim3 PGd = g3(L, L.nx);
  SOLVER_LAUNCH(G, kSB, 0, s, k_pupdate_c<T>)(L.nu, pc.p, pc.z, ctl);
  if (pc.mg.split0) SOLVER_LAUNCH(g3rs(L), kB3, 0, s, k_apply_pq_s<T>)(L, pc.p, pc.q, part, ctl);
  else SOLVER_LAUNCH(g3r(L), kB3, 0, s, k_apply_pq<T>)(L, pc.p, pc.q, part, ctl);
  SOLVER_LAUNCH(G, kSB, 0, s, k_update_rr<T>)(L.nu, pc.d, pc.r, pc.p, pc.q, ctl, part, h_inner, use_graph);
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

// Record the solve of A x = b (x = unknown view of phi) for this instance;
// without programmatic launch edges if a graph holding them cannot be built.
cudaError_t Solver::build_graph(double* x, float* phi32, double phi_c, double phi_a, int nz, double rtol, int maxit) {
  cudaError_t e = build_graph_once(x, phi32, phi_c, phi_a, nz, rtol, maxit);
  if (e != cudaSuccess && g_pdl) {
    g_pdl = false;
    e = build_graph_once(x, phi32, phi_c, phi_a, nz, rtol, maxit);
  }
  return e;
}

cudaError_t Solver::build_graph_once(double* x, float* phi32, double phi_c, double phi_a, int nz, double rtol,
                                     int maxit) {
  if (exec) return cudaSuccess;
  hx = x;
  hphi32 = phi32;
  h_phi_c = phi_c;
  h_phi_a = phi_a;
  h_dphi_dk = (phi_a - phi_c) / (double)nz;
  h_rtol = rtol;
  h_maxit = maxit;
  const char* env = getenv("PIC_SOLVER_GRAPH");
  if (env && env[0] == '0') return cudaSuccess;  // host-driven loop (profilers cannot see conditional graphs)
  cudaStream_t s0 = nullptr;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking))) return e;
  const unsigned long long l0 = g_launches, k0 = g_kernels;
  e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    e = record(s0);
    graph_kernels = g_kernels - k0;
    g_launches = l0;  // recorded, not run
    g_kernels = k0;
    cudaGraph_t whole = nullptr;
    cudaError_t e0 = cudaStreamEndCapture(s0, &whole);
    if (e == cudaSuccess) e = e0;
    graph = whole;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaStreamDestroy(s0);
  if (e != cudaSuccess) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    cudaGetLastError();
  }
  return e;
}

// Add the whole solve (initial norm, outer WHILE node holding the residual, the
// inner WHILE node of PCG iterations and the update) at the capture position of
// s0, in whatever graph s0 is capturing into.
cudaError_t Solver::record(cudaStream_t s0) {
  const Lv L = lv_of(plan[0]);
  const int G = sgrid(L.nu);
  const dim3 PGd = g3(L, L.nx);
  const int mixed = precision != 0;
  const double phi_c = h_phi_c, dphi_dk = h_dphi_dk, rtol = h_rtol;
  const int maxit = h_maxit;
  double* x = hx;
  float* phi32 = hphi32;
  cudaStream_t s1 = aux[0], s2 = aux[1];
  cudaError_t e;
  cudaGraphConditionalHandle h_outer, h_inner;
  cudaGraph_t outer_body = nullptr, inner_body = nullptr;
  if (mixed) {
    SOLVER_LAUNCH(sgrid(L.nu / 4 + 1), kSB, 0, s0, k_dot_bb_ff)(L, f32, fold_first(), fold_last(), part, ctl, rtol, maxit);
  } else {
    SOLVER_LAUNCH(G, kSB, 0, s0, k_dot_bb)(L.nu, b, part, ctl, rtol, maxit);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = add_while(s0, &h_outer, 1u, &outer_body);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s1, outer_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    e = cudaGraphConditionalHandleCreate(&h_inner, outer_body, 0u, 0);
    if (e == cudaSuccess) {
      if (mixed) {
        SOLVER_LAUNCH(g3r(L), kB3, 0, s1, k_residual_ff)(L, phi32, lo32, f32, p32.r, p32.d, phi_c, dphi_dk, part, ctl,
                                                    h_outer, h_inner, inner_rtol, max_outer, 1, (int)p32.mg.split0);
      } else {
        SOLVER_LAUNCH(g3r(L), kB3, 0, s1, k_residual_prep<double>)(L, x, b, ax, p64.r, p64.d, part, ctl, h_outer, h_inner,
                                                              inner_rtol, mixed, max_outer, 1);
      }
    }
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
        SOLVER_LAUNCH(g3(L, L.nx), kB3, 0, s1, k_update_ff)(L, phi32, lo32, p32.d, ctl, (int)p32.mg.split0);
      } else {
        SOLVER_LAUNCH(PGd, kB3, 0, s1, k_axpy_out<double>)(L, x, p64.d, nullptr, phi_c, dphi_dk, ctl);
      }
    }
    cudaGraph_t tmp1;
    cudaError_t e1 = cudaStreamEndCapture(s1, &tmp1);
    if (e == cudaSuccess) e = e1;
  }
  return e;
}

cudaError_t Solver::launch(cudaStream_t s) {
  if (exec) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    // a step being recorded takes the solver's nodes directly (a child graph
    // cannot hold conditional nodes)
    if (cs == cudaStreamCaptureStatusActive) return record(s);
    count_graph(graph_kernels);
    return cudaGraphLaunch(exec, s);
  }
  return run_host(s);
}

// The same kernels driven from the host, one read-back per decision.
cudaError_t Solver::run_host(cudaStream_t s) {
  const Lv L = lv_of(plan[0]);
  const int G = sgrid(L.nu);
  const dim3 PGd = g3(L, L.nx);
  const int mixed = precision != 0;
  const cudaGraphConditionalHandle none = 0;
  auto read = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(host_ctl, ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  };
  if (mixed)
    SOLVER_LAUNCH(sgrid(L.nu / 4 + 1), kSB, 0, s, k_dot_bb_ff)(L, f32, fold_first(), fold_last(), part, ctl, h_rtol,
                                                              h_maxit);
  else SOLVER_LAUNCH(G, kSB, 0, s, k_dot_bb)(L.nu, b, part, ctl, h_rtol, h_maxit);
  for (int outer = 0; outer < max_outer + 1; ++outer) {
    if (mixed)
      SOLVER_LAUNCH(g3r(L), kB3, 0, s, k_residual_ff)(L, hphi32, lo32, f32, p32.r, p32.d, h_phi_c, h_dphi_dk, part, ctl, none,
                                                 none, inner_rtol, max_outer, 0, (int)p32.mg.split0);
    else
      SOLVER_LAUNCH(g3r(L), kB3, 0, s, k_residual_prep<double>)(L, hx, b, ax, p64.r, p64.d, part, ctl, none, none, inner_rtol,
                                                           mixed, max_outer, 0);
    cudaError_t e = read();
    if (e != cudaSuccess) return e;
    const bool go = host_ctl->more != 0;
    while (go) {
      if (mixed) capture_pcg_iteration(p32, L, part, ctl, none, s, 0);
      else capture_pcg_iteration(p64, L, part, ctl, none, s, 0);
      if ((e = read()) != cudaSuccess) return e;
      if (!host_ctl->more) break;
    }
    if (mixed) SOLVER_LAUNCH(g3(L, L.nx), kB3, 0, s, k_update_ff)(L, hphi32, lo32, p32.d, ctl, (int)p32.mg.split0);
    else SOLVER_LAUNCH(PGd, kB3, 0, s, k_axpy_out<double>)(L, hx, p64.d, nullptr, h_phi_c, h_dphi_dk, ctl);
    if (!go) break;
  }
  return cudaGetLastError();
}

cudaError_t Solver::phi64_from_ff(cudaStream_t s) {
  const Lv L = lv_of(plan[0]);
  SOLVER_LAUNCH(g3(L, L.nx), kB3, 0, s, k_phi_from_ff)(L, hphi32, lo32, hx, h_phi_c, h_dphi_dk);
  return cudaGetLastError();
}

cudaError_t Solver::ff_from_phi64(const double* x, cudaStream_t s) {
  const Lv L = lv_of(plan[0]);
  SOLVER_LAUNCH(g3(L, L.nx), kB3, 0, s, k_ff_from_phi)(L, x, hphi32, lo32, h_phi_c, h_dphi_dk);
  return cudaGetLastError();
}

// x was written outside the solver: the next residual takes the stencil.
cudaError_t Solver::invalidate(cudaStream_t s) {
  return cudaMemsetAsync(&ctl->ax_valid, 0, sizeof(int), s);
}

SolveResult Solver::result(cudaStream_t s) {
  cudaMemcpyAsync(host_ctl, ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return result_read();
}

cudaError_t Solver::result_async(cudaStream_t s) {
  return cudaMemcpyAsync(host_ctl, ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s);
}

SolveResult Solver::result_read() const {
  SolveResult r;
  r.iters = host_ctl->it_total;
  r.resid_rel = host_ctl->resid_rel;
  r.converged = host_ctl->converged != 0;
  r.timeout = host_ctl->spec_timeout != 0;
  return r;
}

}  // namespace pic
