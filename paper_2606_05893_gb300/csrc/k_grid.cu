// k_grid.cu -- grid-side kernels: deposition (a3), Poisson right-hand side,
// node field E = -grad phi (a5), fills, host transfer helpers, moments (a11).
#include <algorithm>

#include "pic_internal.cuh"
#include "pic_kernels.cuh"

namespace pic {

constexpr int kBlock = 256;

static int grid_for(long long n, int per_block = kBlock, int max_blocks = 152 * 16) {
  long long b = (n + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// ---------------------------------------------------------------------------
template <class T>
__global__ void k_fill(T* p, long long n, T v) {
  for (long long i = gtid(); i < n; i += gstride()) p[i] = v;
}
void launch_fill64(double* p, long long n, double v, cudaStream_t st) {
  PIC_LAUNCH(grid_for(n), kBlock, 0, st, k_fill<double>)(p, n, v);
}
void launch_fill32(float* p, long long n, float v, cudaStream_t st) {
  PIC_LAUNCH(grid_for(n), kBlock, 0, st, k_fill<float>)(p, n, v);
}
void launch_fill_i32(int32_t* p, long long n, int32_t v, cudaStream_t st) {
  PIC_LAUNCH(grid_for(n), kBlock, 0, st, k_fill<int32_t>)(p, n, v);
}

// ---------------------------------------------------------------------------
// a3: cloud-in-cell deposition. Charged species add q w S / h^3 to the 8
// corner nodes; neutral species add 1 to the count of their cell (NGP).
// Lanes of a warp that sit in the same cell (the store is cell-sorted every
// few steps and particles stay spatially coherent in between) first combine
// their 8 corner weights with shuffles; one lane per cell then issues the 8
// atomics to rho in L2.
// ---------------------------------------------------------------------------
constexpr int kDepBlock = 256;

template <class V>
__device__ __forceinline__ void warp_combine_cell(int cell, V w[8]) {
  const unsigned peers = __match_any_sync(0xffffffffu, cell);
  if (__popc(peers) == 1) return;
  const int leader = __ffs(peers) - 1;
  unsigned rest = peers & ~(1u << leader);
  V acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = w[c];
  while (rest) {
    const int src = __ffs(rest) - 1;
    rest &= rest - 1;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += __shfl_sync(peers, w[c], src);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) w[c] = acc[c];
}

__global__ void __launch_bounds__(kDepBlock) k_deposit_fp64(DepositArgs<Store64> a) {
  const long long n = (long long)a.cnt->n[a.cur][a.species];
  const Grid& g = a.g;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += gstride()) {
    const long long i = base + threadIdx.x;
    const bool valid = i < n;
    int cell = -1;
    long long idx[8];
    double w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (valid) {
      const Particle64 p = store_read(a.st, g, i);
      cell = (int)p.cell;
      corner_nodes(g, p.l.i, p.l.j, p.l.k, idx);
      cic_weights(p.l.fx, p.l.fy, p.l.fz, w);
      const double q = p.pid != kPidDead ? a.qw_h3 * (double)p.mw : 0.0;  // tombstones carry no charge
#pragma unroll
      for (int c = 0; c < 8; ++c) w[c] *= q;
    }
    warp_combine_cell(cell, w);
    const unsigned peers = __match_any_sync(0xffffffffu, cell);
    if (valid && lane == __ffs(peers) - 1) {
#pragma unroll
      for (int c = 0; c < 8; ++c) atomicAdd(&a.rho64[idx[c]], w[c]);
    }
  }
}

__global__ void __launch_bounds__(kDepBlock) k_deposit_mx(DepositArgs<StoreMx> a) {
  const long long n = (long long)a.cnt->n[a.cur][a.species];
  const Grid& g = a.g;
  const float q = (float)a.qw_h3;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += gstride()) {
    const long long i = base + threadIdx.x;
    bool valid = i < n;
    if (valid && !PIC_BOUNDS(a.st.cell[i] >= 0 && a.st.cell[i] < g.ncell, a.cnt)) valid = false;
    int cell = -1;
    float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
      cell = a.st.cell[i];
      cic_weights(a.st.ox[i], a.st.oy[i], a.st.oz[i], w);
      const float qi = a.st.pid[i] != kPidDead ? q * (float)(a.st.mw ? a.st.mw[i] : 1u) : 0.f;  // tombstones carry no charge
#pragma unroll
      for (int c = 0; c < 8; ++c) w[c] *= qi;
    }
    if (warp_run_sum(cell, w) && valid) {
      int ci, cj, ck;
      cell_ijk(g, cell, ci, cj, ck);
      long long idx[8];
      corner_nodes(g, ci, cj, ck, idx);
#pragma unroll
      for (int c = 0; c < 8; ++c) atomicAdd(&a.rho32[idx[c]], w[c]);
    }
  }
}

template <class S>
__global__ void __launch_bounds__(kDepBlock) k_count_neutrals(DepositArgs<S> a) {
  const long long n = (long long)a.cnt->n[a.cur][a.species];
  const Grid& g = a.g;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += gstride()) {
    const long long i = base + threadIdx.x;
    int cell = -1;
    float one[1] = {0.f};  // counts are exact in FP32 (a warp holds 32 at most)
    uint32_t mw = 0u;
    if (i < n) {
      const auto p = store_read(a.st, g, i);
      if (PIC_BOUNDS(particle_cell(p) >= 0 && particle_cell(p) < g.ncell, a.cnt)) {
        cell = (int)particle_cell(p);
        one[0] = p.pid != kPidDead ? 1.f : 0.f;
        mw = p.pid != kPidDead ? p.mw : 0u;
      }
    }
    if (a.st.mw) {  // multiplicities: integer adds per particle (an FP32 run sum could round)
      if (cell >= 0 && mw) atomicAdd(&a.ncount[cell], (int)mw);
    } else if (warp_run_sum(cell, one) && cell >= 0 && one[0] > 0.f) {
      atomicAdd(&a.ncount[cell], (int)one[0]);
    }
  }
}

template <class S>
void launch_deposit(const DepositArgs<S>& a, int grid, cudaStream_t st);
template <>
void launch_deposit<Store64>(const DepositArgs<Store64>& a, int grid, cudaStream_t st) {
  if (a.neutral) PIC_LAUNCH(grid, kDepBlock, 0, st, k_count_neutrals<Store64>)(a);
  else PIC_LAUNCH(grid, kDepBlock, 0, st, k_deposit_fp64)(a);
}
template <>
void launch_deposit<StoreMx>(const DepositArgs<StoreMx>& a, int grid, cudaStream_t st) {
  if (a.neutral) PIC_LAUNCH(grid, kDepBlock, 0, st, k_count_neutrals<StoreMx>)(a);
  else PIC_LAUNCH(grid, kDepBlock, 0, st, k_deposit_mx)(a);
}


// ---------------------------------------------------------------------------
// a4 right-hand side of Eq. (1) scaled by h^2 over the unknown nodes k = 1..nz-1:
//   b = h^2 rho / eps0 (+ phi_c on k = 1) (+ phi_a on k = nz-1)
// ---------------------------------------------------------------------------
// 3-D launch helpers: block (32, 8), x over i, y strided over j, z over planes
// (no integer division in the index math).
static dim3 grid3(const Grid& g, int planes) {
  int gy = (g.ny + 7) / 8;
  gy = gy > 4 ? 4 : gy;
  return dim3((g.nx + 31) / 32, gy, planes);
}
static const dim3 kBlk3(32, 8, 1);

// s = h^2 / eps0, formed once on the host (an FP64 division in every thread
// would queue on the narrow FP64 pipe)
__global__ void __launch_bounds__(256) k_rhs(Grid g, const DevCounters* cnt, const double* __restrict__ rho64,
                                             const float* __restrict__ rho32, double* __restrict__ b, double s) {
  const float s32 = (float)s;
  const int kn = blockIdx.z + 1;  // node plane of this unknown plane
  const int i = blockIdx.x * 32 + threadIdx.x;
  if (i >= g.nx) return;
  const double fold = (kn == 1 ? g.phi_c : 0.0) + (kn == g.nz - 1 ? cnt->anode_V : 0.0);
  for (int j = blockIdx.y * 8 + threadIdx.y; j < g.ny; j += gridDim.y * 8) {
    const long long u = (long long)blockIdx.z * g.nplane + (long long)j * g.nx + i;
    const long long node = u + g.nplane;
    // MIXED: the density is FP32 already; scale it in FP32 and widen once
    double v = rho64 ? s * rho64[node] : (double)(s32 * rho32[node]);
    b[u] = v + fold;
  }
}
void launch_rhs(const Grid& g, const DevCounters* cnt, const double* rho64, const float* rho32, double* b,
                cudaStream_t st) {
  PIC_LAUNCH(grid3(g, g.nz - 1), kBlk3, 0, st, k_rhs)(g, cnt, rho64, rho32, b, g.h * g.h / kEps0);
}

// MIXED path: the FP32 charge term f = fl32(h^2/eps0 rho) over the unknowns,
// without the folded Dirichlet terms (the solver keeps phi relative to the
// vacuum potential). From an FP64 density (a caller's rho) the product is FP64,
// rounded once.
// The unknowns are the nodes of planes 1..nz-1, one contiguous range of the
// node array, so this is a flat pass: four values per thread (16-byte loads)
// where the plane size keeps the range 16-byte aligned.
// The solver keeps phi relative to the vacuum potential of the configured
// electrode voltages; when an external circuit has moved the anode by dV since,
// dV enters as one more folded Dirichlet term on the last unknown plane, and
// the FP32 potential carries dV on the anode plane (the field kernel reads it).
__global__ void __launch_bounds__(256) k_rhs_f32(Grid g, const DevCounters* cnt, const double* __restrict__ rho64,
                                                 const float* __restrict__ rho32, float* __restrict__ f,
                                                 float* __restrict__ phi32, double s) {
  const float s32 = (float)s;
  const long long nu = (long long)(g.nz - 1) * g.nplane;
  const long long last = nu - g.nplane;  // first unknown of the plane next to the anode
  const double dV = cnt->anode_V - g.phi_a;
  const float* r32 = rho32 ? rho32 + g.nplane : nullptr;
  const double* r64 = rho64 ? rho64 + g.nplane : nullptr;
  long long u0 = 0;
  if (r32 && (g.nplane & 3) == 0) {
    const long long n4 = nu >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(r32);
    float4* f4 = reinterpret_cast<float4*>(f);
    const float d4 = (float)dV;
    for (long long q = gtid(); q < n4; q += gstride()) {
      const float4 v = s4[q];
      float4 o = make_float4(s32 * v.x, s32 * v.y, s32 * v.z, s32 * v.w);
      if (dV != 0.0 && (q << 2) >= last) {  // a plane holds whole float4s here
        o.x += d4;
        o.y += d4;
        o.z += d4;
        o.w += d4;
      }
      f4[q] = o;
    }
    u0 = n4 << 2;
  }
  for (long long u = u0 + gtid(); u < nu; u += gstride()) {
    float v = r32 ? s32 * r32[u] : (float)(s * r64[u]);
    if (dV != 0.0 && u >= last) v += (float)dV;
    f[u] = v;
  }
  if (phi32)
    for (long long p = gtid(); p < g.nplane; p += gstride()) phi32[(long long)g.nz * g.nplane + p] = (float)dV;
}
void launch_rhs_f32(const Grid& g, const DevCounters* cnt, const double* rho64, const float* rho32, float* f,
                    float* phi32, cudaStream_t st) {
  PIC_LAUNCH(grid_for((long long)(g.nz - 1) * g.nplane / 4 + 1), kBlock, 0, st, k_rhs_f32)(g, cnt, rho64, rho32, f,
                                                                                          phi32, g.h * g.h / kEps0);
}

__global__ void k_phi_planes(Grid g, const DevCounters* cnt, double* phi) {
  const double va = cnt->anode_V;
  for (long long p = gtid(); p < g.nplane; p += gstride()) {
    phi[p] = g.phi_c;
    phi[(long long)g.nz * g.nplane + p] = va;
  }
}
void launch_phi_planes(const Grid& g, const DevCounters* cnt, double* phi, cudaStream_t st) {
  PIC_LAUNCH(grid_for(g.nplane), kBlock, 0, st, k_phi_planes)(g, cnt, phi);
}

// MIXED: the electrode planes of the FP64 potential as the last solve used them
// (the anode plane of the FP32 deviation holds the circuit's offset dV)
__global__ void k_planes_from_ff(Grid g, const float* __restrict__ phi32, double* __restrict__ phi) {
  const long long top = (long long)g.nz * g.nplane;
  for (long long p = gtid(); p < g.nplane; p += gstride()) {
    phi[p] = g.phi_c;
    phi[top + p] = g.phi_a + (double)phi32[top + p];
  }
}
void launch_planes_from_ff(const Grid& g, const float* phi32, double* phi, cudaStream_t st) {
  PIC_LAUNCH(grid_for(g.nplane), kBlock, 0, st, k_planes_from_ff)(g, phi32, phi);
}

// ---------------------------------------------------------------------------
// a5: node field E = -grad phi. Central differences (periodic in x, y); in z
// central inside, second-order one-sided on the electrode planes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double3 node_field(const Grid& g, const double* __restrict__ f, int i, int j, int k) {
  const long long pl = g.nplane;
  const long long n = (long long)k * pl + (long long)j * g.nx + i;
  const int im = i == 0 ? g.nx - 1 : i - 1, ip = i == g.nx - 1 ? 0 : i + 1;
  const int jm = j == 0 ? g.ny - 1 : j - 1, jp = j == g.ny - 1 ? 0 : j + 1;
  const long long row = n - i;
  const double c = 0.5 * g.inv_h;
  double3 e;
  e.x = (f[row + im] - f[row + ip]) * c;
  e.y = (f[(long long)k * pl + (long long)jm * g.nx + i] - f[(long long)k * pl + (long long)jp * g.nx + i]) * c;
  if (k == 0)
    e.z = (3.0 * f[n] - 4.0 * f[n + pl] + f[n + 2 * pl]) * c;
  else if (k == g.nz)
    e.z = (-3.0 * f[n] + 4.0 * f[n - pl] - f[n - 2 * pl]) * c;
  else
    e.z = (f[n - pl] - f[n + pl]) * c;
  return e;
}

// E.w carries the neutral count of the cell whose lower corner is this node
// (cell and node indices coincide for k < nz), read by the collision filter.
__global__ void __launch_bounds__(256) k_efield64(Grid g, const double* __restrict__ phi, double4_32a* __restrict__ E,
                                                  const int32_t* __restrict__ ncount) {
  const int k = blockIdx.z;
  const int i = blockIdx.x * 32 + threadIdx.x;
  if (i >= g.nx) return;
  for (int j = blockIdx.y * 8 + threadIdx.y; j < g.ny; j += gridDim.y * 8) {
    const long long n = (long long)k * g.nplane + (long long)j * g.nx + i;
    const double3 e = node_field(g, phi, i, j, k);
    double4_32a v;
    v.x = e.x;
    v.y = e.y;
    v.z = e.z;
    v.w = (ncount && k < g.nz) ? (double)ncount[n] : 0.0;
    E[n] = v;
  }
}
void launch_efield64(const Grid& g, const double* phi, double4_32a* E, const int32_t* ncount, cudaStream_t st) {
  PIC_LAUNCH(grid3(g, g.nz + 1), kBlk3, 0, st, k_efield64)(g, phi, E, ncount);
}

// MIXED: E from the FP32 deviation from the vacuum potential, plus the vacuum field
__global__ void __launch_bounds__(256) k_efield32f(Grid g, const float* __restrict__ f, float4* __restrict__ E, float c,
                                                   float ez_vac, const int32_t* __restrict__ ncount) {
  const int k = blockIdx.z;
  const int i = blockIdx.x * 32 + threadIdx.x;
  if (i >= g.nx) return;
  const int pl = (int)g.nplane;
  const int im = i == 0 ? g.nx - 1 : i - 1, ip = i == g.nx - 1 ? 0 : i + 1;
  for (int j = blockIdx.y * 8 + threadIdx.y; j < g.ny; j += gridDim.y * 8) {
    const long long n = (long long)k * pl + (long long)j * g.nx + i;
    const long long row = n - i;
    const int jm = j == 0 ? g.ny - 1 : j - 1, jp = j == g.ny - 1 ? 0 : j + 1;
    const float ex = (f[row + im] - f[row + ip]) * c;
    const float ey = (f[(long long)k * pl + (long long)jm * g.nx + i] - f[(long long)k * pl + (long long)jp * g.nx + i]) * c;
    float ez;
    if (k == 0)
      ez = (3.f * f[n] - 4.f * f[n + pl] + f[n + 2 * pl]) * c;
    else if (k == g.nz)
      ez = (-3.f * f[n] + 4.f * f[n - pl] - f[n - 2 * pl]) * c;
    else
      ez = (f[n - pl] - f[n + pl]) * c;
    E[n] = make_float4(ex, ey, ez + ez_vac, (ncount && k < g.nz) ? (float)ncount[n] : 0.f);
  }
}
void launch_efield32f(const Grid& g, const float* phi32, float4* E, const int32_t* ncount, cudaStream_t st) {
  const float ez_vac = (float)(-(g.phi_a - g.phi_c) / g.Lz);
  PIC_LAUNCH(grid3(g, g.nz + 1), kBlk3, 0, st, k_efield32f)(g, phi32, E, (float)(0.5 * g.inv_h), ez_vac, ncount);
}

// ---------------------------------------------------------------------------
// per-step counter reset
// ---------------------------------------------------------------------------
__global__ void k_step_begin(DevCounters* cnt, StepBegin sb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int s = 0; s < sb.nsp; ++s) cnt->n[sb.out[s]][s] = 0;
  cnt->n_events = 0;
  cnt->n_success = 0;
  cnt->n_success_cx = 0;
  cnt->n_cands = 0;
  cnt->q_cathode_step = 0.0;
  cnt->q_anode_step = 0.0;
}
__global__ void k_step_end(DevCounters* cnt, Circuit c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (c.on) {
    const double dv = (c.dt * (c.V0 - cnt->anode_V) / c.R + cnt->q_anode_step) / c.C;
    cnt->anode_V += dv;
  }
  cnt->step += 1u;
}
void launch_step_end(DevCounters* cnt, const Circuit& c, cudaStream_t st) {
  PIC_LAUNCH(1, 32, 0, st, k_step_end)(cnt, c);
}

void launch_step_begin(DevCounters* cnt, const int* out_buf, int nsp, cudaStream_t st) {
  StepBegin sb;
  sb.nsp = nsp;
  for (int s = 0; s < kMaxSpecies; ++s) sb.out[s] = s < nsp ? out_buf[s] : 0;
  PIC_LAUNCH(1, 1, 0, st, k_step_begin)(cnt, sb);
}

// ---------------------------------------------------------------------------
// host transfer helpers (staging arrays of FP64 x[n][3], v[n][3])
// ---------------------------------------------------------------------------
template <class S>
__global__ void k_load(Grid g, S st, DevCounters* cnt, int cur, int species, long long cap, const double* __restrict__ x,
                       const double* __restrict__ v, const uint32_t* __restrict__ mw, long long n, NextDeposit nd,
                       int neutral) {
  const unsigned long long base = cnt->n[cur][species];
  const uint32_t pid0 = cnt->next_pid;
  for (long long i = gtid(); i < n; i += gstride()) {
    const unsigned long long slot = base + i;
    if (slot >= (unsigned long long)cap) continue;
    store_write(st, g, slot, x[3 * i], x[3 * i + 1], x[3 * i + 2], v[3 * i], v[3 * i + 1], v[3 * i + 2],
                pid0 + (uint32_t)i, mw ? mw[i] : 1u);
    if (nd.on) {  // the next step's deposit is being accumulated: add this particle
      const auto p = store_read(st, g, slot);
      if (neutral) atomicAdd(&nd.ncount[species][cell_now(g, p)], (int)p.mw);
      else if (nd.qw_h3[species] != 0.0) deposit_one(g, p, nd.rho32, nd.rho64, nd.qw_h3[species]);
    }
  }
}
__global__ void k_load_commit(DevCounters* cnt, int cur, int species, long long n, long long cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long m = cnt->n[cur][species] + (unsigned long long)n;
  if (m > (unsigned long long)cap) atomicOr(&cnt->error, ERR_CAPACITY);
  cnt->n[cur][species] = m > (unsigned long long)cap ? (unsigned long long)cap : m;
  cnt->next_pid += (unsigned int)n;
}
template <class S>
void launch_load(const Grid& g, S st, DevCounters* cnt, int cur, int species, long long cap, const double* x,
                 const double* v, const uint32_t* mw, long long n, const NextDeposit& nd, int neutral, cudaStream_t s) {
  if (n <= 0) return;
  PIC_LAUNCH(grid_for(n), kBlock, 0, s, k_load<S>)(g, st, cnt, cur, species, cap, x, v, mw, n, nd, neutral);
  PIC_LAUNCH(1, 1, 0, s, k_load_commit)(cnt, cur, species, n, cap);
}

template <class S>
__global__ void k_download(Grid g, S st, long long n, double* x, double* v, uint32_t* pid, uint32_t* mw) {
  for (long long i = gtid(); i < n; i += gstride()) {
    store_get(st, g, i, x + 3 * i, v + 3 * i, pid + i);
    if (mw) mw[i] = st.mw ? st.mw[i] : 1u;
  }
}
template <class S>
void launch_download(const Grid& g, S st, long long n, double* x, double* v, uint32_t* pid, uint32_t* mw,
                     cudaStream_t s) {
  if (n <= 0) return;
  PIC_LAUNCH(grid_for(n), kBlock, 0, s, k_download<S>)(g, st, n, x, v, pid, mw);
}
template void launch_load<Store64>(const Grid&, Store64, DevCounters*, int, int, long long, const double*,
                                   const double*, const uint32_t*, long long, const NextDeposit&, int, cudaStream_t);
template void launch_load<StoreMx>(const Grid&, StoreMx, DevCounters*, int, int, long long, const double*,
                                   const double*, const uint32_t*, long long, const NextDeposit&, int, cudaStream_t);
template void launch_download<Store64>(const Grid&, Store64, long long, double*, double*, uint32_t*, uint32_t*,
                                       cudaStream_t);
template void launch_download<StoreMx>(const Grid&, StoreMx, long long, double*, double*, uint32_t*, uint32_t*,
                                       cudaStream_t);

// ---------------------------------------------------------------------------
// a2 helpers: sort keys (cell << pid_bits | pid; tombstones sort last) and the
// payload gather through the permutation.
// ---------------------------------------------------------------------------
template <class S>
__global__ void k_cell_keys(Grid g, S st, long long n_max, const unsigned long long* n_dev, int pid_bits,
                            unsigned long long* keys, uint32_t* vals, int32_t* cell_count) {
  const long long n = (long long)*n_dev;
  const unsigned long long pmask = pid_bits >= 32 ? 0xFFFFFFFFull : ((1ull << pid_bits) - 1ull);
  for (long long i = gtid(); i < n && i < n_max; i += gstride()) {
    const auto p = store_read(st, g, i);
    const unsigned long long cell = p.pid == kPidDead ? (unsigned long long)g.ncell : (unsigned long long)particle_cell(p);
    keys[i] = (cell << pid_bits) | ((unsigned long long)p.pid & pmask);
    vals[i] = (uint32_t)i;
    if (cell_count && p.pid != kPidDead) atomicAdd(&cell_count[cell], 1);
  }
}

// Bucket slots of the cell sort: lanes of a warp with the same cell (the store
// is close to cell order between sorts) take consecutive slots with one atomic.
// The loop runs over whole warps, so every lane reaches the match.
template <class S>
__global__ void k_cell_slots(Grid g, S st, long long n_max, const unsigned long long* n_dev, int32_t* cell_count,
                             unsigned long long* __restrict__ words, uint32_t* __restrict__ pids, SegCtl* ctl) {
  const long long n = min((long long)*n_dev, n_max);
  const int lane = threadIdx.x & 31;
  for (long long w0 = gtid() - lane; w0 < n; w0 += gstride()) {
    const long long i = w0 + lane;
    const bool valid = i < n;
    int cell = -1;
    uint32_t pid = 0;
    if (valid) {
      const auto p = store_read(st, g, i);
      pid = p.pid;
      cell = pid == kPidDead ? (int)g.ncell : (int)particle_cell(p);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, cell);
    const int leader = __ffs(peers) - 1;
    int slot0 = 0;
    if (valid && lane == leader)
      slot0 = atomicAdd(cell == (int)g.ncell ? &ctl->dead : &cell_count[cell], __popc(peers));
    slot0 = __shfl_sync(0xffffffffu, slot0, leader);
    if (valid) {
      words[i] = ((unsigned long long)(unsigned)cell << 32) | (unsigned)(slot0 + __popc(peers & ((1u << lane) - 1u)));
      pids[i] = pid;
    }
  }
}
template <class S>
void launch_cell_slots(const Grid& g, S st, long long n_max, const unsigned long long* n_dev, int32_t* cell_count,
                       unsigned long long* words, uint32_t* pids, SegCtl* ctl, cudaStream_t s) {
  PIC_LAUNCH(grid_for(n_max), kBlock, 0, s, k_cell_slots<S>)(g, st, n_max, n_dev, cell_count, words, pids, ctl);
}
template void launch_cell_slots<Store64>(const Grid&, Store64, long long, const unsigned long long*, int32_t*,
                                         unsigned long long*, uint32_t*, SegCtl*, cudaStream_t);
template void launch_cell_slots<StoreMx>(const Grid&, StoreMx, long long, const unsigned long long*, int32_t*,
                                         unsigned long long*, uint32_t*, SegCtl*, cudaStream_t);
template <class S>
void launch_cell_keys(const Grid& g, S st, long long n_max, const unsigned long long* n_dev, int pid_bits,
                      unsigned long long* keys, uint32_t* vals, int32_t* cell_count, cudaStream_t s) {
  PIC_LAUNCH(grid_for(n_max), kBlock, 0, s, k_cell_keys<S>)(g, st, n_max, n_dev, pid_bits, keys, vals, cell_count);
}

__device__ __forceinline__ void copy_slot(const Store64& s, const Store64& d, long long from, long long to) {
  d.x[to] = s.x[from];
  d.y[to] = s.y[from];
  d.z[to] = s.z[from];
  d.vx[to] = s.vx[from];
  d.vy[to] = s.vy[from];
  d.vz[to] = s.vz[from];
  d.pid[to] = s.pid[from];
  if (d.mw) d.mw[to] = s.mw[from];
}
__device__ __forceinline__ void copy_slot(const StoreMx& s, const StoreMx& d, long long from, long long to) {
  d.cell[to] = s.cell[from];
  d.ox[to] = s.ox[from];
  d.oy[to] = s.oy[from];
  d.oz[to] = s.oz[from];
  d.vx[to] = s.vx[from];
  d.vy[to] = s.vy[from];
  d.vz[to] = s.vz[from];
  d.pid[to] = s.pid[from];
  if (d.mw) d.mw[to] = s.mw[from];
}
template <class S>
__global__ void k_gather(S src, S dst, const uint32_t* __restrict__ perm, const unsigned long long* n_dev, long long n_max) {
  const long long n = (long long)*n_dev;
  for (long long i = gtid(); i < n && i < n_max; i += gstride()) copy_slot(src, dst, perm[i], i);
}
template <class S>
void launch_gather(S src, S dst, const uint32_t* perm, const unsigned long long* n_dev, long long n_max,
                   cudaStream_t s) {
  PIC_LAUNCH(grid_for(n_max), kBlock, 0, s, k_gather<S>)(src, dst, perm, n_dev, n_max);
}
template void launch_cell_keys<Store64>(const Grid&, Store64, long long, const unsigned long long*, int,
                                        unsigned long long*, uint32_t*, int32_t*, cudaStream_t);
template void launch_cell_keys<StoreMx>(const Grid&, StoreMx, long long, const unsigned long long*, int,
                                        unsigned long long*, uint32_t*, int32_t*, cudaStream_t);
template void launch_gather<Store64>(Store64, Store64, const uint32_t*, const unsigned long long*, long long,
                                     cudaStream_t);
template void launch_gather<StoreMx>(StoreMx, StoreMx, const uint32_t*, const unsigned long long*, long long,
                                     cudaStream_t);

// after a cell sort into buffer c^1: tombstones (sorted last) are dropped
__global__ void k_sort_commit(DevCounters* cnt, int c, int s) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cnt->n[c ^ 1][s] = cnt->n[c][s] - cnt->n_tomb[s];
  cnt->n_tomb[s] = 0;
}
void launch_sort_commit(DevCounters* cnt, int c, int s, cudaStream_t st) { PIC_LAUNCH(1, 1, 0, st, k_sort_commit)(cnt, c, s); }

// ---------------------------------------------------------------------------
// a11 moments: FP64 reductions (block sums, one atomic per block)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? sm[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Sum of |v|^2 over the live particles of one store. FP64 store: in FP64. Mixed
// store (FP32 velocities): |v|^2 in FP32 (relative rounding ~1e-7, the
// velocities' own precision), summed in FP32 over runs of 8 particles of a
// thread and those partial sums in FP64, so the FP64 pipe (narrow on GB300)
// sees one add per 8 particles instead of seven operations per particle.
__global__ void k_kinetic64(Store64 st, const unsigned long long* n_dev, long long n_max, double* out) {
  const long long n = (long long)*n_dev;
  double acc = 0.0;
  for (long long i = gtid(); i < n && i < n_max; i += gstride())
    if (st.pid[i] != kPidDead) acc += st.vx[i] * st.vx[i] + st.vy[i] * st.vy[i] + st.vz[i] * st.vz[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}
__global__ void k_kinetic_mx(StoreMx st, const unsigned long long* n_dev, long long n_max, double* out) {
  const long long n = min((long long)*n_dev, n_max);
  double acc = 0.0;
  float part = 0.f;
  int run = 0;
  for (long long i = gtid(); i < n; i += gstride()) {
    const float a = st.vx[i], b = st.vy[i], c = st.vz[i];
    if (st.pid[i] != kPidDead) part += fmaf(a, a, fmaf(b, b, c * c));
    if (++run == 8) {
      acc += (double)part;
      part = 0.f;
      run = 0;
    }
  }
  acc += (double)part;
  acc = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}
// Variable weights: sum of mw |v|^2 into out[0] and of mw into out[1] (both in
// FP64, |v|^2 from the stored velocities).
__device__ __forceinline__ double stored_v2(const Store64& st, long long i) {
  return st.vx[i] * st.vx[i] + st.vy[i] * st.vy[i] + st.vz[i] * st.vz[i];
}
__device__ __forceinline__ double stored_v2(const StoreMx& st, long long i) {
  const double a = st.vx[i], b = st.vy[i], c = st.vz[i];
  return a * a + b * b + c * c;
}
template <class S>
__global__ void k_kinetic_w(S st, const unsigned long long* n_dev, long long n_max, double* out_v2, double* out_m) {
  const long long n = min((long long)*n_dev, n_max);
  double acc = 0.0, m = 0.0;
  for (long long i = gtid(); i < n; i += gstride()) {
    if (st.pid[i] == kPidDead) continue;
    const double w = (double)st.mw[i];
    acc += w * stored_v2(st, i);
    m += w;
  }
  acc = block_sum(acc);
  __syncthreads();  // block_sum's shared buffer is reused
  m = block_sum(m);
  if (threadIdx.x == 0) {
    atomicAdd(out_v2, acc);
    atomicAdd(out_m, m);
  }
}
template <class S>
void launch_kinetic_w(S st, const unsigned long long* n_dev, long long n_max, double* out_v2, double* out_m,
                      cudaStream_t s) {
  PIC_LAUNCH(grid_for(n_max), kBlock, 0, s, k_kinetic_w<S>)(st, n_dev, n_max, out_v2, out_m);
}
template void launch_kinetic_w<Store64>(Store64, const unsigned long long*, long long, double*, double*, cudaStream_t);
template void launch_kinetic_w<StoreMx>(StoreMx, const unsigned long long*, long long, double*, double*, cudaStream_t);

template <class S>
void launch_kinetic(S st, const unsigned long long* n_dev, long long n_max, double* out, cudaStream_t s);
template <>
void launch_kinetic<Store64>(Store64 st, const unsigned long long* n_dev, long long n_max, double* out, cudaStream_t s) {
  PIC_LAUNCH(grid_for(n_max), kBlock, 0, s, k_kinetic64)(st, n_dev, n_max, out);
}
template <>
void launch_kinetic<StoreMx>(StoreMx st, const unsigned long long* n_dev, long long n_max, double* out, cudaStream_t s) {
  PIC_LAUNCH(grid_for(n_max), kBlock, 0, s, k_kinetic_mx)(st, n_dev, n_max, out);
}

// Sum over edges of (delta phi)^2. A block takes whole node rows (k, j) and its
// threads the nodes i of a row, so the row's indices cost one division per row
// rather than two 64-bit divisions per node.
__global__ void k_field_energy(Grid g, const double* __restrict__ f, double* out) {
  const long long pl = g.nplane;
  const long long rows = (long long)g.ny * (g.nz + 1);
  double acc = 0.0;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int k = (int)(r / g.ny);
    const int j = (int)(r - (long long)k * g.ny);
    const double* row = f + (long long)k * pl + (long long)j * g.nx;
    const double* north = f + (long long)k * pl + (long long)(j + 1 == g.ny ? 0 : j + 1) * g.nx;
    const bool up = k < g.nz;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const double c = row[i];
      const double dx = row[i + 1 == g.nx ? 0 : i + 1] - c;
      const double dy = north[i] - c;
      acc += dx * dx + dy * dy;
      if (up) {
        const double dz = row[pl + i] - c;
        acc += dz * dz;
      }
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}
void launch_field_energy(const Grid& g, const double* phi, double* out, cudaStream_t s) {
  const long long rows = (long long)g.ny * (g.nz + 1);
  const int threads = g.nx >= 256 ? 256 : (g.nx >= 128 ? 128 : 64);
  const int grid = (int)std::min<long long>(rows, 152 * 16);
  PIC_LAUNCH(grid, threads, 0, s, k_field_energy)(g, phi, out);
}

// MIXED: the same sum from the solver's own state, without rebuilding phi in
// FP64: phi = phi_c on the cathode plane, phi_a + d on the anode plane (d: the
// external circuit's offset in the FP32 deviation's anode plane) and
// vac(k) + hi + lo in between (vac linear in k, hi the FP32 deviation, lo its
// FP32 remainder). The vacuum part cancels in x and y and is one constant per
// z edge (dz_in inside, dz_top for the last edge). A difference of two exact
// FP32 values is rounded relative to the difference itself, so every edge
// difference comes out within ~1e-7 of its size; the squares are summed in
// FP32 over runs of 8 nodes and those sums in FP64.
__global__ void k_field_energy_ff(Grid g, const float* __restrict__ hi, const float* __restrict__ lo, float dz_in,
                                  float dz_top, double* out) {
  // threads (x over a row, y over kFeRows rows): a block keeps that many rows'
  // loads in flight at once
  const long long pl = g.nplane;
  const long long rows = (long long)g.ny * (g.nz + 1);
  double acc = 0.0;
  float part = 0.f;
  int run = 0;
  for (long long r = (long long)blockIdx.x * blockDim.y + threadIdx.y; r < rows; r += (long long)gridDim.x * blockDim.y) {
    const int k = (int)(r / g.ny);
    const int j = (int)(r - (long long)k * g.ny);
    const long long c0 = (long long)j * g.nx;                               // row j in a plane
    const long long cn = (long long)(j + 1 == g.ny ? 0 : j + 1) * g.nx;     // row j + 1
    const float* H = hi + (long long)k * pl;                                 // plane k (node view)
    const float* L = lo + (long long)(k - 1) * pl;                           // plane k (unknown view)
    const bool interior = k > 0 && k < g.nz;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const int ip = i + 1 == g.nx ? 0 : i + 1;
      float h0 = 0.f, hx = 0.f, hy = 0.f, l0 = 0.f, lx = 0.f, ly = 0.f;
      if (k > 0) {
        h0 = H[c0 + i];
        hx = H[c0 + ip];
        hy = H[cn + i];
      }
      if (interior) {
        l0 = L[c0 + i];
        lx = L[c0 + ip];
        ly = L[cn + i];
      }
      const float dx = (hx - h0) + (lx - l0);
      const float dy = (hy - h0) + (ly - l0);
      float sq = fmaf(dx, dx, dy * dy);
      if (k < g.nz) {
        const float h1 = H[pl + c0 + i];
        const float l1 = k + 1 < g.nz ? L[pl + c0 + i] : 0.f;
        const float dz = (k + 1 == g.nz ? dz_top : dz_in) + ((h1 - h0) + (l1 - l0));
        sq = fmaf(dz, dz, sq);
      }
      part += sq;
      if (++run == 8) {
        acc += (double)part;
        part = 0.f;
        run = 0;
      }
    }
  }
  acc += (double)part;
  // block sum over the linear thread index (two-dimensional block)
  __shared__ double sm[32];
  const int t = threadIdx.y * blockDim.x + threadIdx.x, nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((t & 31) == 0) sm[t >> 5] = acc;
  __syncthreads();
  if (t < 32) {
    acc = t < nw ? sm[t] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (t == 0) atomicAdd(out, acc);
  }
}
void launch_field_energy_ff(const Grid& g, const float* phi32, const float* lo32, double* out, cudaStream_t s) {
  const double dphi_dk = (g.phi_a - g.phi_c) / (double)g.nz;
  const float dz_in = (float)dphi_dk;
  const float dz_top = (float)(g.phi_a - (g.phi_c + dphi_dk * (double)(g.nz - 1)));
  const long long rows = (long long)g.ny * (g.nz + 1);
  const int tx = g.nx >= 128 ? 128 : (g.nx >= 64 ? 64 : 32);
  const int ty = 256 / tx;
  const int grid = (int)std::min<long long>((rows + ty - 1) / ty, 152 * 8);
  PIC_LAUNCH(grid, dim3(tx, ty), 0, s, k_field_energy_ff)(g, phi32, lo32, dz_in, dz_top, out);
}

// The moments of the mixed store in one launch: every block sums |v|^2 of its
// share of every species (four particles per pass in FP32, the passes in FP64),
// then its share of the field energy's node rows (as k_field_energy_ff), and
// writes its totals to a.part; the last block to finish adds the blocks'
// totals in block order (a sum that does not depend on timing) into out
// (out[sp] per species, out[16] the field).
__global__ void k_moments_mx(MomentsMx a, double* out) {
  __shared__ double sm[32];
  const int t = threadIdx.x, nw = blockDim.x >> 5;
  auto block_total = [&](double v) -> double {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) sm[t >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (t < 32) {
      r = t < nw ? sm[t] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();  // sm is reused by the next total
    return r;
  };
  {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int sp = 0; sp < a.nsp; ++sp) {
      const float* __restrict__ vx = a.st[sp].vx;
      const float* __restrict__ vy = a.st[sp].vy;
      const float* __restrict__ vz = a.st[sp].vz;
      const uint32_t* __restrict__ pid = a.st[sp].pid;
      const long long n = min((long long)*a.n_dev[sp], a.n_max[sp]);
      double acc = 0.0;
      // four particles per pass (their loads in flight together), summed in FP32,
      // the pass sums in FP64
      for (long long i = (long long)blockIdx.x * blockDim.x + t; i < n; i += 4 * stride) {
        float part = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const long long ii = i + q * stride;
          if (ii < n) {
            const float x = __ldg(vx + ii), y = __ldg(vy + ii), z = __ldg(vz + ii);
            if (__ldg(pid + ii) != kPidDead) part += fmaf(x, x, fmaf(y, y, z * z));
          }
        }
        acc += (double)part;
      }
      acc = block_total(acc);
      if (t == 0) a.part[(long long)blockIdx.x * kMomSlots + sp] = acc;
    }
  }
  // field energy: edge differences of the solver's FP32 hi / lo state, rows of
  // nodes over (blocks - kin_blocks) blocks, several rows per block at once
  const Grid& g = a.g;
  const long long pl = g.nplane;
  const long long rows = (long long)g.ny * (g.nz + 1);
  const int tx = a.fe_tx, ty = blockDim.x / tx, lx0 = t % tx, ly0 = t / tx;
  const long long fb = blockIdx.x, nfb = gridDim.x;
  // the squared edge differences at node (i, row r); rows of the same thread
  // are taken two at a time so that their loads are in flight together
  auto node_sq = [&](long long r, int i) -> float {
    const int k = (int)r / g.ny;  // rows < 2^31
    const int j = (int)r - k * g.ny;
    const long long c0 = (long long)j * g.nx;
    const long long cn = (long long)(j + 1 == g.ny ? 0 : j + 1) * g.nx;
    const float* H = a.hi + (long long)k * pl;
    const float* L = a.lo + (long long)(k - 1) * pl;
    const bool interior = k > 0 && k < g.nz;
    const int ip = i + 1 == g.nx ? 0 : i + 1;
    float h0 = 0.f, hx = 0.f, hy = 0.f, l0 = 0.f, lxv = 0.f, ly = 0.f, h1 = 0.f, l1 = 0.f;
    if (k > 0) {
      h0 = H[c0 + i];
      hx = H[c0 + ip];
      hy = H[cn + i];
    }
    if (interior) {
      l0 = L[c0 + i];
      lxv = L[c0 + ip];
      ly = L[cn + i];
    }
    if (k < g.nz) h1 = H[pl + c0 + i];
    if (k + 1 < g.nz) l1 = L[pl + c0 + i];
    const float dx = (hx - h0) + (lxv - l0);
    const float dy = (hy - h0) + (ly - l0);
    float sq = fmaf(dx, dx, dy * dy);
    if (k < g.nz) {
      const float dz = (k + 1 == g.nz ? a.dz_top : a.dz_in) + ((h1 - h0) + (l1 - l0));
      sq = fmaf(dz, dz, sq);
    }
    return sq;
  };
  double acc = 0.0;
  const long long rstep = nfb * ty;
  for (long long r = fb * ty + ly0; r < rows; r += 2 * rstep) {
    const bool two = r + rstep < rows;
    for (int i = lx0; i < g.nx; i += tx) {
      const float s0 = node_sq(r, i);
      const float s1 = two ? node_sq(r + rstep, i) : 0.f;
      acc += (double)(s0 + s1);
    }
  }
  acc = block_total(acc);
  if (t == 0) a.part[(long long)blockIdx.x * kMomSlots + kMaxSpecies] = acc;
  // the last block: every block's totals are written
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int q = 0; q <= a.nsp; ++q) {
    const int slot = q < a.nsp ? q : kMaxSpecies;
    double v = 0.0;
    for (int b = t; b < (int)gridDim.x; b += blockDim.x) v += a.part[(long long)b * kMomSlots + slot];
    v = block_total(v);
    if (t == 0) out[q < a.nsp ? q : 16] = v;
  }
  if (t == 0) *a.ticket = 0u;
}
void launch_moments_mx(const MomentsMx& a0, double* out, cudaStream_t s) {
  MomentsMx a = a0;
  const Grid& g = a.g;
  const double dphi_dk = (g.phi_a - g.phi_c) / (double)g.nz;
  a.dz_in = (float)dphi_dk;
  a.dz_top = (float)(g.phi_a - (g.phi_c + dphi_dk * (double)(g.nz - 1)));
  a.fe_tx = g.nx >= 128 ? 128 : (g.nx >= 64 ? 64 : 32);
  a.kin_blocks = 0;
  // one wave: every block resident at once (the blocks' shares are equal, so a
  // second partial wave would take as long as the first)
  static int grid = 0;
  if (grid == 0) {
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_moments_mx, kBlock, 0);
    grid = std::max(1, std::min(kMomBlocks, occ * sms));
  }
  PIC_LAUNCH(grid, kBlock, 0, s, k_moments_mx)(a, out);
}

// Philox on the device (test hook)
__global__ void k_philox(long long n, uint4 ctr, uint2 key, uint32_t* out) {
  for (long long i = gtid(); i < n; i += gstride()) {
    const uint4 r = philox(make_uint4(ctr.x + (uint32_t)i, ctr.y, ctr.z, ctr.w), key);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
  }
}
void launch_philox(long long n, uint4 ctr, uint2 key, uint32_t* out, cudaStream_t s) {
  PIC_LAUNCH(grid_for(n), kBlock, 0, s, k_philox)(n, ctr, key, out);
}

}  // namespace pic
