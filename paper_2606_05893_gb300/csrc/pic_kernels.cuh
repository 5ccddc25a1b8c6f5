// pic_kernels.cuh -- particle views, kernel argument blocks and launcher
// declarations shared by the kernel translation units and the host runtime.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// cell location (FP64 store): g = x * (1/h), cell = floor(g) clamped, fraction g - cell
// ---------------------------------------------------------------------------
struct Loc {
  int i, j, k;
  double fx, fy, fz;
};

__device__ __forceinline__ Loc locate64(const Grid& g, double x, double y, double z) {
  Loc l;
  const double gx = x * g.inv_h, gy = y * g.inv_h, gz = z * g.inv_h;
  int i = (int)floor(gx), j = (int)floor(gy), k = (int)floor(gz);
  i = min(max(i, 0), g.nx - 1);
  j = min(max(j, 0), g.ny - 1);
  k = min(max(k, 0), g.nz - 1);
  l.i = i;
  l.j = j;
  l.k = k;
  l.fx = gx - i;
  l.fy = gy - j;
  l.fz = gz - k;
  return l;
}

// The 8 node indices of cell (i,j,k), periodic in i and j: order (a,b,c) with
// a fastest, node = (k+c, j+b, i+a).
__device__ __forceinline__ void corner_nodes(const Grid& g, int i, int j, int k, long long idx[8]) {
  const int i1 = i + 1 == g.nx ? 0 : i + 1;
  const int j1 = j + 1 == g.ny ? 0 : j + 1;
  const long long pl = g.nplane;
  const long long r00 = (long long)k * pl + (long long)j * g.nx;
  const long long r10 = (long long)k * pl + (long long)j1 * g.nx;
  idx[0] = r00 + i;
  idx[1] = r00 + i1;
  idx[2] = r10 + i;
  idx[3] = r10 + i1;
  idx[4] = r00 + pl + i;
  idx[5] = r00 + pl + i1;
  idx[6] = r10 + pl + i;
  idx[7] = r10 + pl + i1;
}

template <class T>
__device__ __forceinline__ void cic_weights(T fx, T fy, T fz, T w[8]) {
  const T wx0 = T(1) - fx, wy0 = T(1) - fy, wz0 = T(1) - fz;
  w[0] = wx0 * wy0 * wz0;
  w[1] = fx * wy0 * wz0;
  w[2] = wx0 * fy * wz0;
  w[3] = fx * fy * wz0;
  w[4] = wx0 * wy0 * fz;
  w[5] = fx * wy0 * fz;
  w[6] = wx0 * fy * fz;
  w[7] = fx * fy * fz;
}

__device__ __forceinline__ void cell_ijk(const Grid& g, int cell, int& i, int& j, int& k) {
  const int t = fdiv(cell, g.fdx);
  i = cell - t * g.nx;
  k = fdiv(t, g.fdy);
  j = t - k * g.ny;
}

// Runs of equal keys among consecutive lanes (a cell-sorted store keeps the
// particles of a cell together): sums each run's values into its first lane
// (suffix sums bounded by the run's last lane, five shuffle steps) and returns
// true there. Equal keys that are not adjacent form separate runs. Every lane
// of the warp must call it.
template <int N>
__device__ __forceinline__ bool warp_run_sum(int key, float (&w)[N]) {
  const int lane = threadIdx.x & 31;
  const int next = __shfl_down_sync(0xffffffffu, key, 1);
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  const unsigned tail = __ballot_sync(0xffffffffu, lane == 31 || next != key);
  const int run_end = lane + __ffs(tail >> lane) - 1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int c = 0; c < N; ++c) {
      const float t = __shfl_down_sync(0xffffffffu, w[c], o);
      if (lane + o <= run_end) w[c] += t;
    }
  }
  return lane == 0 || prev != key;
}

// ---------------------------------------------------------------------------
// particle views
// ---------------------------------------------------------------------------
struct Particle64 {
  double x, y, z, vx, vy, vz;
  uint32_t pid;
  uint32_t mw;     // multiplicity (1 without variable weights)
  long long cell;  // cell at read time (x^n)
  Loc l;
  float nc;        // neutral count of the cell (4th component of the node field)

  template <class A>
  __device__ __forceinline__ double3 gather(const Grid& g, const A& a) {
    long long idx[8];
    corner_nodes(g, l.i, l.j, l.k, idx);
    double w[8];
    cic_weights(l.fx, l.fy, l.fz, w);
    double3 e = make_double3(0.0, 0.0, 0.0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double4_32a en = a.E64[idx[c]];
      e.x += w[c] * en.x;
      e.y += w[c] * en.y;
      e.z += w[c] * en.z;
      if (c == 0) nc = (float)en.w;
    }
    return e;
  }
  template <class A>
  __device__ __forceinline__ void kick(const A& a, const double3& e) {
    vx += a.qm_dt * e.x;
    vy += a.qm_dt * e.y;
    vz += a.qm_dt * e.z;
  }
  // x^{n+1} = x^n + v dt; returns -1 (z < 0), +1 (z >= Lz) or 0 (inside, x/y wrapped)
  __device__ __forceinline__ int drift(const Grid& g) {
    const double xn = x + vx * g.dt, yn = y + vy * g.dt, zn = z + vz * g.dt;
    if (zn < 0.0) return -1;
    if (zn >= g.Lz) return 1;
    x = wrap_coord(xn, g.Lx, g.inv_Lx);
    y = wrap_coord(yn, g.Ly, g.inv_Ly);
    z = zn;
    return 0;
  }
  // where the straight path x^n -> x^{n+1} crosses z = 0 (after drift returned
  // -1, which leaves x^n in place): x^n - v z^n / vz
  __device__ __forceinline__ void cathode_point(const Grid& g, double& xc, double& yc) const {
    const double f = z / vz;
    xc = wrap_coord(x - vx * f, g.Lx, g.inv_Lx);
    yc = wrap_coord(y - vy * f, g.Ly, g.inv_Ly);
  }
  __device__ __forceinline__ double3 vel() const { return make_double3(vx, vy, vz); }
  __device__ __forceinline__ double v2() const { return vx * vx + vy * vy + vz * vz; }
  __device__ __forceinline__ float v2f() const { return (float)v2(); }
  // isotropic elastic scattering at constant speed (FP64, as the oracle):
  // cos theta = 2 U1 - 1, phi = 2 pi U2 from Philox(pid, step, TAG_SCATTER)
  __device__ __forceinline__ void scatter_isotropic(const uint4& d) {
    const double ct = 2.0 * u01_64(d.x, d.y) - 1.0;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    const double ph = 2.0 * kPi * u01_64(d.z, d.w);
    const double uu = sqrt(v2());
    set_v(uu * st * cos(ph), uu * st * sin(ph), uu * ct);
  }
  __device__ __forceinline__ void set_v(double a, double b, double c) {
    vx = a;
    vy = b;
    vz = c;
  }
  __device__ __forceinline__ void scale_v(double s) {
    vx *= s;
    vy *= s;
    vz *= s;
  }
};

struct ParticleMx {
  int32_t cell;
  float ox, oy, oz, vx, vy, vz;
  uint32_t pid;
  uint32_t mw;     // multiplicity (1 without variable weights)
  float nc;  // neutral count of the cell (4th component of the node field)

  template <class A>
  __device__ __forceinline__ float3 gather(const Grid& g, const A& a) {
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    long long idx[8];
    corner_nodes(g, i, j, k, idx);
    float w[8];
    cic_weights(ox, oy, oz, w);
    float3 e = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float4 en = __ldg(&a.E32[idx[c]]);
      e.x = fmaf(w[c], en.x, e.x);
      e.y = fmaf(w[c], en.y, e.y);
      e.z = fmaf(w[c], en.z, e.z);
      if (c == 0) nc = en.w;
    }
    return e;
  }
  template <class A>
  __device__ __forceinline__ void kick(const A& a, const float3& e) {
    vx = fmaf(a.qm_dt_f, e.x, vx);
    vy = fmaf(a.qm_dt_f, e.y, vy);
    vz = fmaf(a.qm_dt_f, e.z, vz);
  }
  // offset += v dt / h; whole cells move the integer index (periodic in x, y).
  // floor(o) without conversions: adding 1.5 2^23 rounds o to an integer in the
  // float's mantissa (|o| < 2^22), read back as an int, then corrected down.
  __device__ __forceinline__ static int split(float& o) {
    if (!(fabsf(o) < 4194304.f)) {  // far outside any cell step: conversion path
      const float f = floorf(o);
      o -= f;
      return (int)f;
    }
    const float t = o + 12582912.f;
    float f = t - 12582912.f;
    int d = __float_as_int(t) - 0x4B400000;
    if (f > o) {
      f -= 1.f;
      d -= 1;
    }
    o -= f;
    if (o >= 1.f) {
      o -= 1.f;
      d += 1;
    }
    return d;
  }
  __device__ __forceinline__ int drift(const Grid& g) {
    ox = fmaf(vx, g.dt_over_h_f, ox);
    oy = fmaf(vy, g.dt_over_h_f, oy);
    oz = fmaf(vz, g.dt_over_h_f, oz);
    const int di = split(ox), dj = split(oy), dk = split(oz);
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    k += dk;
    if (k < 0) {
      // absorbed at the cathode: keep x^{n+1} for the hit log (cell of the
      // wrapped column in plane 0, oz = z^{n+1} / h < 0)
      i = fwrap(i + di, g.fdx);
      j = fwrap(j + dj, g.fdy);
      cell = j * g.nx + i;
      oz += (float)k;
      return -1;
    }
    if (k >= g.nz) return 1;
    i = fwrap(i + di, g.fdx);
    j = fwrap(j + dj, g.fdy);
    cell = (k * g.ny + j) * g.nx + i;
    return 0;
  }
  // where the straight path x^n -> x^{n+1} crosses z = 0 (after drift returned -1)
  __device__ __forceinline__ void cathode_point(const Grid& g, double& xc, double& yc) const {
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    const double f = (double)oz * g.h / (double)vz;  // z^{n+1} / vz, z^{n+1} < 0 and vz < 0
    xc = wrap_coord(((double)i + (double)ox) * g.h - (double)vx * f, g.Lx, g.inv_Lx);
    yc = wrap_coord(((double)j + (double)oy) * g.h - (double)vy * f, g.Ly, g.inv_Ly);
  }
  __device__ __forceinline__ double3 vel() const { return make_double3(vx, vy, vz); }
  __device__ __forceinline__ double v2() const {
    return (double)vx * (double)vx + (double)vy * (double)vy + (double)vz * (double)vz;
  }
  __device__ __forceinline__ float v2f() const { return fmaf(vx, vx, fmaf(vy, vy, vz * vz)); }
  // the same scattering in FP32 from the same draws: cos theta = U1 - (1 - U1)
  // and sin theta = 2 sqrt(U1 (1 - U1)) with U1 and 1 - U1 each rounded once
  // from FP64 (no cancellation near the poles), phi = 2 pi U2 via sincospif.
  __device__ __forceinline__ void scatter_isotropic(const uint4& d) {
    const double U1 = u01_64(d.x, d.y);
    const float a = (float)U1, b = (float)(1.0 - U1);
    const float ct = a - b, st = 2.f * sqrtf(a * b);
    float sp, cp;
    sincospif(2.f * (float)u01_64(d.z, d.w), &sp, &cp);
    const float uu = sqrtf(v2f());
    vx = uu * st * cp;
    vy = uu * st * sp;
    vz = uu * ct;
  }
  __device__ __forceinline__ void set_v(double a, double b, double c) {
    vx = (float)a;
    vy = (float)b;
    vz = (float)c;
  }
  __device__ __forceinline__ void scale_v(double s) {
    const float f = (float)s;
    vx *= f;
    vy *= f;
    vz *= f;
  }
};

// Add the 8 CIC weights w of cell (i, j, k) to an FP32 node grid. Each of the
// four (j, k) rows takes its two x-neighbours with one 16-byte vector reduction
// (red.global.add.v4.f32, zeros in the other lanes) when they share an aligned
// float4 (nx a multiple of 4, so rows start 16-byte aligned, and no periodic
// wrap): one L2 request instead of two. Otherwise two scalar atomics.
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}
__device__ __forceinline__ void cic_add_f32(float* rho, const Grid& g, int i, int j, int k, const float w[8],
                                            bool vec_rows) {
  const int i1 = i + 1 == g.nx ? 0 : i + 1;
  const int j1 = j + 1 == g.ny ? 0 : j + 1;
  const int a4 = i & ~3, off = i - a4;
  const bool vec = vec_rows && i1 == i + 1 && off < 3;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int jj = (r & 1) ? j1 : j;
    const int kk = k + (r >> 1);
    float* row = rho + ((long long)kk * g.ny + jj) * g.nx;
    const float wa = w[2 * r], wb = w[2 * r + 1];
    if (vec) {
      const float v0 = off == 0 ? wa : 0.f;
      const float v1 = off == 1 ? wa : (off == 0 ? wb : 0.f);
      const float v2 = off == 2 ? wa : (off == 1 ? wb : 0.f);
      const float v3 = off == 2 ? wb : 0.f;
      red_add_v4(row + a4, v0, v1, v2, v3);
    } else {
      atomicAdd(row + i, wa);
      atomicAdd(row + i1, wb);
    }
  }
}

// One particle's CIC charge (q = charge * weight / h^3) at its stored position,
// plain atomics (injection and ionization: few particles), and its cell.
__device__ __forceinline__ void deposit_one(const Grid& g, const ParticleMx& p, float* rho32, double* rho64, double q) {
  (void)rho64;
  float w[8];
  cic_weights(p.ox, p.oy, p.oz, w);
  int i, j, k;
  cell_ijk(g, p.cell, i, j, k);
  long long idx[8];
  corner_nodes(g, i, j, k, idx);
  const float qf = (float)q * (float)p.mw;
#pragma unroll
  for (int c = 0; c < 8; ++c) atomicAdd(&rho32[idx[c]], w[c] * qf);
}
__device__ __forceinline__ void deposit_one(const Grid& g, const Particle64& p, float* rho32, double* rho64, double q) {
  (void)rho32;
  const Loc l = locate64(g, p.x, p.y, p.z);
  double w[8];
  cic_weights(l.fx, l.fy, l.fz, w);
  long long idx[8];
  corner_nodes(g, l.i, l.j, l.k, idx);
  const double qm = q * (double)p.mw;
#pragma unroll
  for (int c = 0; c < 8; ++c) atomicAdd(&rho64[idx[c]], w[c] * qm);
}
__device__ __forceinline__ int cell_now(const Grid& g, const ParticleMx& p) {
  (void)g;
  return p.cell;
}
__device__ __forceinline__ int cell_now(const Grid& g, const Particle64& p) {
  const Loc l = locate64(g, p.x, p.y, p.z);
  return (l.k * g.ny + l.j) * g.nx + l.i;
}

// Accumulation of the next step's charge density and neutral counts while the
// particles are at hand (push, injection, ionization): the deposit of step n+1
// is then ready when it starts.
struct NextDeposit {
  int on;                        // accumulate (0: the next step deposits from scratch)
  float* rho32;                  // MIXED
  double* rho64;                 // FP64
  int32_t* ncount[kMaxSpecies];  // neutral species
  double qw_h3[kMaxSpecies];     // charge * weight / h^3 per species
};

template <class S>
struct PTraits;
template <>
struct PTraits<Store64> {
  using P = Particle64;
  static constexpr int kMinBlocks = 2;  // resident 256-thread push blocks per SM
};
template <>
struct PTraits<StoreMx> {
  using P = ParticleMx;
  static constexpr int kMinBlocks = 4;
};

__device__ __forceinline__ Particle64 store_read(const Store64& s, const Grid& g, long long i) {
  Particle64 p;
  p.x = s.x[i];
  p.y = s.y[i];
  p.z = s.z[i];
  p.vx = s.vx[i];
  p.vy = s.vy[i];
  p.vz = s.vz[i];
  p.pid = s.pid[i];
  p.mw = s.mw ? s.mw[i] : 1u;
  p.l = locate64(g, p.x, p.y, p.z);
  p.cell = ((long long)p.l.k * g.ny + p.l.j) * g.nx + p.l.i;
  return p;
}
__device__ __forceinline__ ParticleMx store_read(const StoreMx& s, const Grid& g, long long i) {
  ParticleMx p;
  p.cell = s.cell[i];
  p.ox = s.ox[i];
  p.oy = s.oy[i];
  p.oz = s.oz[i];
  p.vx = s.vx[i];
  p.vy = s.vy[i];
  p.vz = s.vz[i];
  p.pid = s.pid[i];
  p.mw = s.mw ? s.mw[i] : 1u;
  return p;
}
__device__ __forceinline__ long long particle_cell(const Particle64& p) { return p.cell; }
__device__ __forceinline__ long long particle_cell(const ParticleMx& p) { return p.cell; }

__device__ __forceinline__ void store_write_p(const Store64& s, long long i, const Particle64& p) {
  s.x[i] = p.x;
  s.y[i] = p.y;
  s.z[i] = p.z;
  s.vx[i] = p.vx;
  s.vy[i] = p.vy;
  s.vz[i] = p.vz;
  s.pid[i] = p.pid;
  if (s.mw) s.mw[i] = p.mw;
}
__device__ __forceinline__ void store_write_p(const StoreMx& s, long long i, const ParticleMx& p) {
  s.cell[i] = p.cell;
  s.ox[i] = p.ox;
  s.oy[i] = p.oy;
  s.oz[i] = p.oz;
  s.vx[i] = p.vx;
  s.vy[i] = p.vy;
  s.vz[i] = p.vz;
  s.pid[i] = p.pid;
  if (s.mw) s.mw[i] = p.mw;
}
__device__ __forceinline__ void store_write_v(const Store64& s, long long i, const Particle64& p) {
  s.vx[i] = p.vx;
  s.vy[i] = p.vy;
  s.vz[i] = p.vz;
}
__device__ __forceinline__ void store_write_v(const StoreMx& s, long long i, const ParticleMx& p) {
  s.vx[i] = p.vx;
  s.vy[i] = p.vy;
  s.vz[i] = p.vz;
}
__device__ __forceinline__ void store_kill(const Store64& s, long long i) { s.pid[i] = kPidDead; }
__device__ __forceinline__ void store_kill(const StoreMx& s, long long i) { s.pid[i] = kPidDead; }

// Write from FP64 values (injection, host upload).
__device__ __forceinline__ void store_write(const Store64& s, const Grid& g, long long i, double x, double y, double z,
                                            double vx, double vy, double vz, uint32_t pid, uint32_t mw = 1u) {
  (void)g;
  if (s.mw) s.mw[i] = mw;
  s.x[i] = x;
  s.y[i] = y;
  s.z[i] = z;
  s.vx[i] = vx;
  s.vy[i] = vy;
  s.vz[i] = vz;
  s.pid[i] = pid;
}
__device__ __forceinline__ float offset_of(double gcoord, int cell) {
  float o = (float)(gcoord - (double)cell);
  if (o >= 1.f) o = 0x1.fffffep-1f;
  if (o < 0.f) o = 0.f;
  return o;
}
__device__ __forceinline__ void store_write(const StoreMx& s, const Grid& g, long long i, double x, double y, double z,
                                            double vx, double vy, double vz, uint32_t pid, uint32_t mw = 1u) {
  if (s.mw) s.mw[i] = mw;
  const Loc l = locate64(g, x, y, z);
  s.cell[i] = (l.k * g.ny + l.j) * g.nx + l.i;
  s.ox[i] = offset_of(x * g.inv_h, l.i);
  s.oy[i] = offset_of(y * g.inv_h, l.j);
  s.oz[i] = offset_of(z * g.inv_h, l.k);
  s.vx[i] = (float)vx;
  s.vy[i] = (float)vy;
  s.vz[i] = (float)vz;
  s.pid[i] = pid;
}
// Read as FP64 values (host download).
__device__ __forceinline__ void store_get(const Store64& s, const Grid& g, long long i, double* x, double* v,
                                          uint32_t* pid) {
  (void)g;
  x[0] = s.x[i];
  x[1] = s.y[i];
  x[2] = s.z[i];
  v[0] = s.vx[i];
  v[1] = s.vy[i];
  v[2] = s.vz[i];
  *pid = s.pid[i];
}
__device__ __forceinline__ void store_get(const StoreMx& s, const Grid& g, long long i, double* x, double* v,
                                          uint32_t* pid) {
  int ci, cj, ck;
  cell_ijk(g, s.cell[i], ci, cj, ck);
  x[0] = ((double)ci + (double)s.ox[i]) * g.h;
  x[1] = ((double)cj + (double)s.oy[i]) * g.h;
  x[2] = ((double)ck + (double)s.oz[i]) * g.h;
  v[0] = s.vx[i];
  v[1] = s.vy[i];
  v[2] = s.vz[i];
  *pid = s.pid[i];
}

// ---------------------------------------------------------------------------
// argument blocks
// ---------------------------------------------------------------------------
struct McArgs {
  int nch;
  XsDev ch[kMaxXsec];
  const int32_t* ncount[kMaxXsec];  // neutral counts of each channel's target
  double dens[kMaxXsec];            // w_target / h^3
  float bound_f[kMaxXsec];          // (max sigma) w_target / h^3, FP32 filter
  float dens_f[kMaxXsec];           // dens rounded to FP32 (FP32 enclosure of Eq. 4)
  double half_m_over_e;             // E_eV = v^2 m / (2 e)
  float half_m_over_e_f;
  float bg_density_f;
  double mass;
  uint2 key;
  int bg_mode;  // fixed background density (test mode)
  double bg_density;
  int count_in_field;  // all channels share one target: its cell count rides in E.w
};

struct StepBegin {
  int nsp;
  int out[kMaxSpecies];
};

struct InjSrc {
  int species;
  double cx, cy, R, sig;
};

template <class S>
struct InjectArgs {
  Grid g;
  DevCounters* cnt;
  S st[kMaxSpecies];
  int cur[kMaxSpecies];
  long long cap[kMaxSpecies];
  int nsrc;
  InjSrc src[kMaxSources];
  InjectPlan* plan;  // sources and carries (device); the launch's last block advances the carries
  uint2 key;
  NextDeposit nd;
  int role[kMaxSpecies];
  int nsp;
};

// Surface-coupling output: ions absorbed at the cathode (n == nullptr: not
// logged for this species). n counts every hit; the first cap are stored.
struct HitLog {
  unsigned long long* n;
  long long cap;
  uint32_t* pid;
  int32_t* species;
  uint32_t* step;
  double* xy;  // 2 per hit: crossing point of z = 0
  double* v;   // 3 per hit: v^{n+1/2}
};

template <class S>
struct PushArgs {
  Grid g;
  DevCounters* cnt;
  S in, out;
  int cur_in, species;
  long long cap;
  double qm_dt;
  float qm_dt_f;
  double mass, weight, charge;
  const double4_32a* E64;
  const float4* E32;
  McArgs mc;
  Event* ev;
  int ev_cap;
  int32_t* ev_head;
  Cand* cand;
  uint32_t* cand_cell;
  int cand_cap;
  int32_t* cand_head;
  NextDeposit nd;
  HitLog hits;
};

struct ResolveArgs {
  DevCounters* cnt;
  Event* ev;
  int ev_cap;
  int32_t* ev_head;
  Cand* cand;
  uint32_t* cand_cell;  // cell of each candidate (a flat array the rank kernel scans)
  int cand_cap;
  int32_t* cand_head;
  unsigned long long* sort_keys;
  uint32_t* sort_vals;
};

// Buffers and capacities the resolve commit updates (species < 0: absent).
struct ResolveCommit {
  int e_out, e_sp;
  long long e_cap;
  int i_out, i_sp;
  long long i_cap;
  int n_out, n_sp;
  long long n_cap;
  int ev_cap;
  int weighted;  // variable weights: partial conversions, 3 pids per successful event
};

template <class S>
struct ApplyArgs {
  Grid g;
  DevCounters* cnt;
  const Event* ev;
  int ev_cap;
  const Cand* cand;
  int cand_cap;
  const uint32_t* sorted_vals;
  XsDev ch[kMaxXsec];
  uint2 key;
  S e_st;                  // ionization: electrons (e_species < 0 without an ionization channel)
  int e_out, e_species;
  long long e_cap;
  double e_mass;
  S n_st;                  // the target neutrals (victims; exchanged ions land here)
  int n_out;
  long long n_cap;
  S i_st;                  // the ions (victims land here; exchanging ions leave)
  int i_out, i_species;
  long long i_cap;
  uint32_t* log;
  NextDeposit nd;
  int n_species;
  int32_t* ev_head;      // per-cell list heads, emptied for the next step
  int32_t* cand_head;
  ResolveCommit commit;  // applied by the launch's last block
};


template <class S>
struct DepositArgs {
  Grid g;
  DevCounters* cnt;
  S st;
  int cur, species;
  int neutral;       // 1: count into ncount, 0: charge into rho
  double qw_h3;      // q w / h^3
  double* rho64;
  float* rho32;
  int32_t* ncount;
};

// ---------------------------------------------------------------------------
// launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------
template <class S>
void launch_inject(const InjectArgs<S>& a, int grid, cudaStream_t st);
void launch_step_end(DevCounters* cnt, const Circuit& c, cudaStream_t st);
template <class S>
void launch_push(const PushArgs<S>& a, int role, bool mcc, int grid, cudaStream_t st);
void launch_resolve_rank(const ResolveArgs& a, int grid, cudaStream_t st);
template <class S>
void launch_resolve_apply(const ApplyArgs<S>& a, int grid, cudaStream_t st);

template <class S>
void launch_deposit(const DepositArgs<S>& a, int grid, cudaStream_t st);
void launch_fill64(double* p, long long n, double v, cudaStream_t st);
void launch_fill32(float* p, long long n, float v, cudaStream_t st);
void launch_fill_i32(int32_t* p, long long n, int32_t v, cudaStream_t st);
void launch_rhs(const Grid& g, const DevCounters* cnt, const double* rho64, const float* rho32, double* b,
                cudaStream_t st);
void launch_rhs_f32(const Grid& g, const DevCounters* cnt, const double* rho64, const float* rho32, float* f,
                    float* phi32, cudaStream_t st);
void launch_efield64(const Grid& g, const double* phi, double4_32a* E, const int32_t* ncount, cudaStream_t st);
void launch_efield32f(const Grid& g, const float* phi32, float4* E, const int32_t* ncount, cudaStream_t st);
void launch_phi_planes(const Grid& g, const DevCounters* cnt, double* phi, cudaStream_t st);
void launch_planes_from_ff(const Grid& g, const float* phi32, double* phi, cudaStream_t st);
void launch_step_begin(DevCounters* cnt, const int* out_buf, int nsp, cudaStream_t st);

template <class S>
void launch_load(const Grid& g, S st, DevCounters* cnt, int cur, int species, long long cap, const double* x,
                 const double* v, const uint32_t* mw, long long n, const NextDeposit& nd, int neutral, cudaStream_t s);
template <class S>
void launch_download(const Grid& g, S st, long long n, double* x, double* v, uint32_t* pid, uint32_t* mw,
                     cudaStream_t s);

template <class S>
void launch_cell_keys(const Grid& g, S st, long long n_max, const unsigned long long* n_dev, int pid_bits,
                      unsigned long long* keys, uint32_t* vals, int32_t* cell_count, cudaStream_t s);

// radix sort of (u64 key, u32 value) pairs over bits [bit0, bit1); n read from
// the device (at most n_max). Returns 0 if the result is in (ka, va), 1 if in (kb, vb).
// a2 cell sort by buckets (k_sort.cu, k_grid.cu): every particle takes a slot in
// its cell's bucket (warp-aggregated atomics on the cell counts, so the order
// inside a bucket is arbitrary), the buckets are laid out by a scan of the
// counts, and each bucket is then sorted by (pid, input index), which makes the
// permutation the unique one of the key (cell, pid). Dead slots form a last
// bucket after every cell, in input order. A bucket larger than kSegBig sets
// `overflow`, and the caller sorts that species by the radix path instead.
struct SegCtl {
  int dead;      // slots taken in the dead bucket
  int nmid;      // buckets of kSegSmall < m <= kSegMid entries, listed from the front of `big`
  int nbig;      // buckets of kSegMid < m entries, listed from the back of `big`
  int overflow;  // a bucket of more than kSegBig entries
};
constexpr int kSegSmall = 16;   // sorted by one thread
constexpr int kSegMid = 256;    // by one warp
constexpr int kSegBig = 4096;   // by one block
template <class S>
void launch_cell_slots(const Grid& g, S st, long long n_max, const unsigned long long* n_dev, int32_t* cell_count,
                       unsigned long long* words, uint32_t* pids, SegCtl* ctl, cudaStream_t s);
void launch_seg_scatter(long long ncell, long long n_max, const unsigned long long* n_dev,
                        const unsigned long long* words, const uint32_t* pids, const long long* cell_start,
                        unsigned long long* out, uint32_t* perm, cudaStream_t s);
void launch_seg_sort(long long ncell, const long long* cell_start, const unsigned long long* n_dev,
                     const unsigned long long* vals, uint32_t* perm, int32_t* big, SegCtl* ctl, cudaStream_t s);

struct SortBuffers {
  unsigned long long *ka, *kb;
  uint32_t *va, *vb;
  uint32_t* hist;      // 256 * nblocks(n_max)
  uint32_t* digit_tot; // 256
  int* small_done;     // set when the single-block path sorted the input
  long long n_max;
  cudaStream_t aux;    // capture stream of the radix passes inside a recorded step (small path)
};
long long sort_hist_entries(long long n_max);
int radix_sort_pairs(const SortBuffers& b, const unsigned long long* n_dev, int bit0, int bit1, cudaStream_t s,
                     bool small_path = false);
// exclusive scan of int32 counts[n] into int64 out[n+1] (out[n] = total)
size_t scan_temp_bytes(long long n);
void exclusive_scan_i32_i64(const int32_t* counts, long long n, long long* out, void* temp, cudaStream_t s);
template <class S>
void launch_gather(S src, S dst, const uint32_t* perm, const unsigned long long* n_dev, long long n_max,
                   cudaStream_t s);

void launch_sort_commit(DevCounters* cnt, int c, int s, cudaStream_t st);

// moments
template <class S>
void launch_kinetic(S st, const unsigned long long* n_dev, long long n_max, double* out, cudaStream_t s);
void launch_field_energy(const Grid& g, const double* phi, double* out, cudaStream_t s);
void launch_field_energy_ff(const Grid& g, const float* phi32, const float* lo32, double* out, cudaStream_t s);
// every species' sum of |v|^2 (out[sp]) and the field energy sum (out[16]) of the
// mixed store in one launch (written, not added to); part holds kMomBlocks x
// kMomSlots doubles, ticket one counter that is 0 between launches
constexpr int kMomBlocks = 152 * 8;
constexpr int kMomSlots = kMaxSpecies + 1;
struct MomentsMx {
  Grid g;
  int nsp;
  StoreMx st[kMaxSpecies];
  const unsigned long long* n_dev[kMaxSpecies];
  long long n_max[kMaxSpecies];
  const float* hi;  // the solver's FP32 state at nodes
  const float* lo;  // and its low part over the unknowns
  double* part;
  unsigned int* ticket;
  float dz_in, dz_top;   // set by the launcher
  int fe_tx, kin_blocks; // set by the launcher (kin_blocks unused: every block takes both parts)
};
void launch_moments_mx(const MomentsMx& a, double* out, cudaStream_t s);
template <class S>
void launch_kinetic_w(S st, const unsigned long long* n_dev, long long n_max, double* out_v2, double* out_m,
                      cudaStream_t s);

void launch_philox(long long n, uint4 ctr, uint2 key, uint32_t* out, cudaStream_t s);

}  // namespace pic
