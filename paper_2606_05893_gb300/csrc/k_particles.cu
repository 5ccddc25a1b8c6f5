// k_particles.cu -- particle kernels of the PIC/MCC step (FP64 and MIXED stores).
//
//   a1 inject            k_inject<Store>
//   a5+a6+a7+a8 (+a10)   k_push<Store>: field gather at x^n, leapfrog kick/drift,
//                        absorption at the electrodes, Monte Carlo collisions
//                        (Eq. 4), warp-aggregated compaction into the other buffer
//   a9 ionization and    k_resolve_rank / k_resolve_apply (with the commit and the list-head reset)
//      charge exchange
//
// Collision test (Eq. 4): P = 1 - exp(-u dt sum_c n_c sigma_c(E)), decided with the
// FP64 uniform U1 of Philox(pid, step, TAG_MCC). Because 1 - exp(-x) <= x and
// sigma_c(E) <= max sigma_c, every electron whose FP32 draw exceeds an FP32 upper
// bound of x (with a safety margin) cannot collide; only the remainder (a fraction
// of about P of the electrons) evaluates P and the channel choice exactly in FP64.
#include "pic_internal.cuh"
#include "pic_kernels.cuh"

namespace pic {

constexpr int kPushBlock = 256;
constexpr int kPushWarps = kPushBlock / 32;
constexpr int kIlp = 2;  // particles per thread and round

// ---------------------------------------------------------------------------
// cross sections
// ---------------------------------------------------------------------------
// Exact FP64 lookup: bisection for E_lo <= E < E_hi, then the interpolation
// sigma_lo + t (sigma_hi - sigma_lo), t = (E - E_lo)/(E_hi - E_lo).
__device__ double xs_sigma64(const XsDev& c, double E) {
  if (!(E > c.thr)) return 0.0;
  if (c.n == 1) return c.sig[0];
  if (E <= c.E[0]) return c.sig[0];
  if (E >= c.E[c.n - 1]) return c.sig[c.n - 1];
  int lo = 0, hi = c.n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (E < c.E[mid]) hi = mid; else lo = mid;
  }
  const double t = (E - c.E[lo]) / (c.E[lo + 1] - c.E[lo]);
  return c.sig[lo] + t * (c.sig[lo + 1] - c.sig[lo]);
}

// Exact FP64 collision test of Eq. (4); returns -1 (none) or the channel slot.
__device__ int mcc_exact_dt(const McArgs& m, long long cell, double v2, double U, double dt) {
  const double u = sqrt(v2);
  const double E = m.half_m_over_e * v2;
  double cum[kMaxXsec];
  double nu = 0.0;
  for (int a = 0; a < m.nch; ++a) {
    const double nt = m.bg_mode ? m.bg_density : (double)m.ncount[a][cell] * m.dens[a];
    nu += nt * xs_sigma64(m.ch[a], E);
    cum[a] = nu;
  }
  if (!(nu > 0.0)) return -1;
  const double P = -expm1(-u * dt * nu);
  if (!(U < P)) return -1;
  int a = 0;
  while (a < m.nch - 1 && !(U < P * (cum[a] / nu))) ++a;
  return a;
}

// FP32 filter, first part: sum_a n_a max sigma_a of the cell (0 when the cell
// holds no target, and then nu = 0 in FP64 too: no collision, no draw). cnt0 >= 0
// is the target count of the cell taken from the node field (all channels share
// that target); otherwise the counts are read per channel.
__device__ __forceinline__ float mcc_nu_bound(const McArgs& m, long long cell, float cnt0) {
  float nb = 0.f;
  for (int a = 0; a < m.nch; ++a) {
    const float cnt = m.bg_mode ? 1.f : (cnt0 >= 0.f ? cnt0 : (float)m.ncount[a][cell]);
    nb = fmaf(cnt, m.bound_f[a], nb);
  }
  return nb;
}
// Second part: true when the electron certainly does not collide, since
// x_upper = u dt nb >= x >= P (1.001 covers FP32 rounding) and U32 is within
// 2^-24 of the FP64 draw.
__device__ __forceinline__ bool mcc_cannot_collide(float nb, float v2f, float U32, float dt_f) {
  const float xu = sqrtf(v2f) * dt_f * nb * 1.001f;
  return U32 - 0x1p-24f > xu;
}

// ---------------------------------------------------------------------------
// FP32 enclosure of the FP64 decision
// ---------------------------------------------------------------------------
// The FP32 energy E32 = (m/2e) v^2 is within a relative 8 2^-24 = 2^-21 of the
// FP64 energy E. When E32 is farther than kBrk = 2^-18 (relative) from every
// breakpoint of the piecewise-linear table (threshold, first and last point,
// table points), E lies on the same linear piece as E32 and sigma(E) is inside
// [lo, hi] below; otherwise the enclosure is not attempted (returns false).
constexpr float kBrk = 0x1p-18f;
constexpr float kRel = 0x1p-18f;  // relative margin for FP32 rounding of products and sums

__device__ __forceinline__ bool xs_sigma32(const XsDev& c, float E32, float& lo, float& hi) {
  const float band = kBrk * E32;
  if (c.thr_f > 0.f) {
    if (E32 + band <= c.thr_f) {  // certainly E <= thr
      lo = hi = 0.f;
      return true;
    }
    if (E32 - band < c.thr_f) return false;
  } else if (!(E32 > 1e-30f)) {
    return false;
  }
  float s0, sl = 0.f;
  if (c.n == 1) {
    s0 = c.sigf[0];
  } else if (E32 + band <= c.Ef[0]) {
    s0 = c.sigf[0];
  } else if (E32 - band >= c.Ef[c.n - 1]) {
    s0 = c.sigf[c.n - 1];
  } else {
    if (E32 - band < c.Ef[0] || E32 + band > c.Ef[c.n - 1]) return false;
    // bucket of ln E32 (floor without a float->int conversion), then a short scan
    float v = (__logf(E32) - c.lnE0) * c.inv_dln;
    v = fminf(fmaxf(v, 0.f), (float)(kXsBuckets - 1));
    const float t = v + 12582912.f;
    int b = __float_as_int(t) - 0x4B400000;
    if (t - 12582912.f > v) --b;
    int k = c.bucket[b];
    while (k > 0 && c.Ef[k] > E32) --k;
    while (k < c.n - 2 && c.Ef[k + 1] <= E32) ++k;
    const float e0 = c.Ef[k], e1 = c.Ef[k + 1];
    if (E32 - e0 < band || e1 - E32 < band) return false;
    sl = c.slopef[k];
    s0 = fmaf(E32 - e0, sl, c.sigf[k]);
    const float err = kRel * (fabsf(c.sigf[k]) + fabsf(sl) * E32);
    lo = s0 - err;
    hi = s0 + err;
    return true;
  }
  lo = s0 * (1.f - kRel);
  hi = s0 * (1.f + kRel);
  return true;
}

// The channel the FP64 rule of Eq. (4) would pick (mcc_exact_dt), decided in
// FP32: -1 none, a >= 0 channel, -2 undecided (U within the rounding band of a
// threshold, or E near a table breakpoint): the caller then runs the FP64 rule.
// With x = u dt nu, the FP64 rule compares U with T_a = P cum_a / nu
// = g(x) u dt cum_a, g(x) = (1 - e^-x)/x, and 1 - x/2 <= g(x) <= 1 - x/2 + x^2/6
// for x >= 0. Each T_a is enclosed from the sigma enclosures, the FP32 draw is
// within 2^-24 of the FP64 one.
__device__ int mcc_decide32(const McArgs& m, long long cell, float v2f, float U32, float dt_f, float cnt0) {
  const float E32 = m.half_m_over_e_f * v2f;
  const float ud = sqrtf(v2f) * dt_f;
  float slo[kMaxXsec], shi[kMaxXsec];
  float clo = 0.f, chi = 0.f;
  for (int a = 0; a < m.nch; ++a) {
    const float na = m.bg_mode ? m.bg_density_f
                               : (cnt0 >= 0.f ? cnt0 : (float)m.ncount[a][cell]) * m.dens_f[a];
    float lo, hi;
    if (!xs_sigma32(m.ch[a], E32, lo, hi)) return -2;
    clo = fmaf(na, fmaxf(lo, 0.f), clo);
    chi = fmaf(na, hi, chi);
    slo[a] = clo;
    shi[a] = chi;
  }
  const float xlo = ud * clo * (1.f - kRel), xhi = ud * chi * (1.f + kRel);
  const float glo = 1.f - 0.5f * xhi;
  const float ghi = 1.f - 0.5f * xlo + xhi * xhi * (1.f / 6.f) * (1.f + kRel);
  const float Ulo = U32 - 0x1p-24f, Uhi = U32 + 0x1p-24f;
  for (int a = 0; a < m.nch; ++a) {
    const float Tlo = glo * ud * slo[a] * (1.f - kRel);
    const float Thi = ghi * ud * shi[a] * (1.f + kRel);
    if (Uhi < Tlo) return a;
    if (!(Ulo >= Thi)) return -2;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// a1: injection
// ---------------------------------------------------------------------------
// -2 log U in FP32 for the Box-Muller radius, accurate to about 1e-7 relative
// over all of (0, 1): U from the 53-bit draw, and near 1 through log1p of the
// exactly formed 1 - U (log of a rounded U would lose 1 - U there)
__device__ __forceinline__ float m2log_u(uint32_t a, uint32_t b) {
  const double u = u01_64(a, b);
  return u < 0.5 ? -2.f * logf((float)u) : -2.f * log1pf(-(float)(1.0 - u));
}

// This step's counts from the carry accumulators (FP64, the host formula:
// acc += mu; n = floor(acc); acc -= n): first particle of each source, its
// offset among its species' new particles, and the total.
struct InjCounts {
  long long first[kMaxSources + 1];
  long long offset[kMaxSources];
  long long add[kMaxSpecies];
  double acc[kMaxSources];
};
__device__ __forceinline__ void inject_counts(const InjectPlan& P, InjCounts& c) {
  long long total = 0;
  for (int s = 0; s < kMaxSpecies; ++s) c.add[s] = 0;
  for (int q = 0; q < P.nsrc; ++q) {
    double acc = P.acc[q] + P.mu[q];
    const double nf = floor(acc);
    acc -= nf;
    c.acc[q] = acc;
    const long long n = (long long)nf;
    c.first[q] = total;
    c.offset[q] = c.add[P.species[q]];
    c.add[P.species[q]] += n;
    total += n;
  }
  c.first[P.nsrc] = total;
}

// a1 in one launch: every block forms the step's counts from the carries (the
// same FP64 arithmetic in each), places its share of the new particles, and the
// last block to finish commits the step (carries, store counts, next pid).
template <class S>
__global__ void k_inject(InjectArgs<S> a) {
  __shared__ InjCounts sc;
  __shared__ bool s_last;
  const InjectPlan& P = *a.plan;
  if (threadIdx.x == 0) inject_counts(P, sc);
  __syncthreads();
  const long long total = sc.first[P.nsrc];
  const uint32_t step = a.cnt->step;
  // particle t on block t mod G (thread t / G): a step injects tens to hundreds of
  // particles, each with FP64 transcendentals, and one SM's narrow FP64 pipe
  // would take them all one after another; spread this way each SM gets one or two
  for (long long t = blockIdx.x + (long long)gridDim.x * threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    // source of this particle
    int q = 0;
    while (q + 1 < a.nsrc && t >= sc.first[q + 1]) ++q;
    const InjSrc& s = a.src[q];
    const long long kth = t - sc.first[q];
    const uint32_t pid = a.cnt->next_pid + (uint32_t)t;
    const unsigned long long base = a.cnt->n[a.cur[s.species]][s.species];
    const unsigned long long slot = base + sc.offset[q] + kth;
    if (slot >= (unsigned long long)a.cap[s.species]) {
      atomicOr(&a.cnt->error, ERR_CAPACITY);
      continue;
    }
    const uint4 dp = draw(a.key, pid, step, TAG_INJ_POS);
    const uint4 d1 = draw(a.key, pid, step, TAG_INJ_VXY);
    const uint4 d2 = draw(a.key, pid, step, TAG_INJ_VZ);
    const uint4 d3 = draw(a.key, pid, step, TAG_INJ_Z);
    double x, y, z, vx, vy, vz;
    if constexpr (std::is_same<S, StoreMx>::value) {
      // the FP32 store takes FP32 velocity samples (FP64 transcendentals run on
      // the narrow FP64 pipe): the same 53-bit uniforms rounded to FP32
      // (relative error 2^-24), the same formulas in FP32. The position stays
      // FP64: the source radius spans many cells, and an FP32 r cos(theta)
      // would be far coarser than the store's FP32 offset within a cell.
      double sr, cr;
      float s1, c1;
      sincospi(2.0 * u01_64(dp.z, dp.w), &sr, &cr);
      const double r = s.R * sqrt(u01_64(dp.x, dp.y));
      x = wrap_coord(s.cx + r * cr, a.g.Lx, a.g.inv_Lx);
      y = wrap_coord(s.cy + r * sr, a.g.Ly, a.g.inv_Ly);
      sincospif(2.f * (float)u01_64(d1.z, d1.w), &s1, &c1);
      const float rad1 = sqrtf(m2log_u(d1.x, d1.y));
      const float n3 = sqrtf(m2log_u(d2.x, d2.y)) * cospif(2.f * (float)u01_64(d2.z, d2.w));
      const float sig = (float)s.sig;
      vx = (double)(sig * (rad1 * c1));
      vy = (double)(sig * (rad1 * s1));
      vz = (double)(sig * fabsf(n3));
      z = (double)((float)u01_64(d3.x, d3.y) * (float)vz * (float)a.g.dt);
    } else {
      const double r = s.R * sqrt(u01_64(dp.x, dp.y));
      const double th = 2.0 * kPi * u01_64(dp.z, dp.w);
      x = wrap_coord(s.cx + r * cos(th), a.g.Lx, a.g.inv_Lx);
      y = wrap_coord(s.cy + r * sin(th), a.g.Ly, a.g.inv_Ly);
      const double rad1 = sqrt(-2.0 * log(u01_64(d1.x, d1.y)));
      const double ph1 = 2.0 * kPi * u01_64(d1.z, d1.w);
      const double n1 = rad1 * cos(ph1), n2 = rad1 * sin(ph1);
      const double n3 = sqrt(-2.0 * log(u01_64(d2.x, d2.y))) * cos(2.0 * kPi * u01_64(d2.z, d2.w));
      vx = s.sig * n1;
      vy = s.sig * n2;
      vz = s.sig * fabs(n3);
      z = u01_64(d3.x, d3.y) * vz * a.g.dt;
    }
    store_write(a.st[s.species], a.g, slot, x, y, z, vx, vy, vz, pid);
    if (a.nd.on) {  // the next step's deposit is being accumulated: add this particle
      const auto p = store_read(a.st[s.species], a.g, slot);
      if (a.role[s.species] == ROLE_NEUTRAL) atomicAdd(&a.nd.ncount[s.species][cell_now(a.g, p)], 1);
      else if (a.nd.qw_h3[s.species] != 0.0) deposit_one(a.g, p, a.nd.rho32, a.nd.rho64, a.nd.qw_h3[s.species]);
    }
  }
  // the last block: every block's reads of the counters and carries are done
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.plan->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  InjectPlan& W = *a.plan;
  for (int q = 0; q < W.nsrc; ++q) W.acc[q] = sc.acc[q];
  W.ticket = 0u;
  if (total == 0) return;
  for (int sp = 0; sp < a.nsp; ++sp) {
    if (sc.add[sp] == 0) continue;
    unsigned long long nn = a.cnt->n[a.cur[sp]][sp] + sc.add[sp];
    if (nn > (unsigned long long)a.cap[sp]) nn = a.cap[sp];
    a.cnt->injected[sp] += nn - a.cnt->n[a.cur[sp]][sp];
    a.cnt->n[a.cur[sp]][sp] = nn;
  }
  a.cnt->next_pid += (unsigned int)total;
}

// ---------------------------------------------------------------------------
// a5-a8 + a10: gather / push / absorb / collide / compact
// ---------------------------------------------------------------------------
// Next-step deposit from the push. MIXED store: the lanes of a warp whose
// particles landed in the same cell are grouped with __match_any_sync (adjacent
// or not: the particles of one cell are interleaved with those of the next
// plane after a drift), the group's lowest lane adds the others' CIC weights
// from shared memory and issues the group's reductions: one per row and group.
// The neutral count likewise (the group's size). FP64 store: plain FP64
// atomics (summing doubles across lanes would load the narrow FP64 pipe).
// Every lane of the warp calls it.
template <bool CHARGED, bool NEUTRAL>
__device__ __forceinline__ void next_deposit(const PushArgs<StoreMx>& a, const ParticleMx& p, bool stored) {
  const int lane = threadIdx.x & 31;
  // a lane without a particle gets a key of its own (negative: never a cell)
  const int key = stored ? p.cell : -1 - lane;
  const unsigned grp = __match_any_sync(0xffffffffu, key);
  const bool lead = stored && (__ffs(grp) - 1) == lane;
  if (CHARGED) {
    // this warp's weights, [corner][lane] (conflict-free rows of 32 words)
    __shared__ float s_w[kPushWarps][8 * 32];
    float* sw = s_w[threadIdx.x >> 5];
    float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (stored) {
      cic_weights(p.ox, p.oy, p.oz, w);
      const float q = (float)a.nd.qw_h3[a.species] * (float)p.mw;
#pragma unroll
      for (int c = 0; c < 8; ++c) w[c] *= q;
    }
    if (__ballot_sync(0xffffffffu, grp != (1u << lane))) {  // some lanes share a cell
#pragma unroll
      for (int c = 0; c < 8; ++c) sw[c * 32 + lane] = w[c];
      __syncwarp();
      if (lead) {
        for (unsigned m = grp & ~(1u << lane); m; m &= m - 1) {
          const int l = __ffs(m) - 1;
#pragma unroll
          for (int c = 0; c < 8; ++c) w[c] += sw[c * 32 + l];
        }
      }
      __syncwarp();  // the buffer is refilled by the next call
    }
    if (lead) {
      int i, j, k;
      cell_ijk(a.g, key, i, j, k);
      cic_add_f32(a.nd.rho32, a.g, i, j, k, w, (a.g.nx & 3) == 0);
    }
  }
  if (NEUTRAL) {
    if (a.in.mw == nullptr) {
      if (lead) atomicAdd(&a.nd.ncount[a.species][key], __popc(grp));
    } else if (stored) {
      atomicAdd(&a.nd.ncount[a.species][key], (int)p.mw);  // multiplicities
    }
  }
}
template <bool CHARGED, bool NEUTRAL>
__device__ __forceinline__ void next_deposit(const PushArgs<Store64>& a, const Particle64& p, bool stored) {
  if (!stored) return;
  if (CHARGED) deposit_one(a.g, p, nullptr, a.nd.rho64, a.nd.qw_h3[a.species]);
  if (NEUTRAL) atomicAdd(&a.nd.ncount[a.species][cell_now(a.g, p)], (int)p.mw);
}

// One ion absorbed at the cathode into the hit log (rare: out of the push's
// main path; scalar arguments, so the particle stays in registers).
__device__ __noinline__ void log_cathode_hit(const HitLog& h, uint32_t pid, int species, uint32_t step, double xc,
                                             double yc, double vx, double vy, double vz) {
  const unsigned long long k = atomicAdd(h.n, 1ull);
  if (k >= (unsigned long long)h.cap) return;
  h.pid[k] = pid;
  h.species[k] = species;
  h.step[k] = step;
  h.xy[2 * k] = xc;
  h.xy[2 * k + 1] = yc;
  h.v[3 * k] = vx;
  h.v[3 * k + 1] = vy;
  h.v[3 * k + 2] = vz;
}

template <class S, bool CHARGED, bool MCC, bool NEUTRAL>
__global__ void __launch_bounds__(kPushBlock, PTraits<S>::kMinBlocks) k_push(PushArgs<S> a) {
  // Each thread advances kIlp particles per round (their loads are issued
  // together, so the memory latency of one hides behind the others). Output
  // slots are reserved once per block and round (one global atomic per
  // kIlp * 256 particles); absorption statistics and elastic counts accumulate
  // in shared memory and reach HBM once per block.
  __shared__ unsigned int s_wcnt[kPushWarps];
  __shared__ unsigned long long s_base;
  // per-thread tallies, each touched by its own thread only (no atomics, no
  // registers held): absorbed at cathode / anode, their sum of v^2, elastic
  // collisions; reduced once per block at the end
  // (with variable weights v^2 is weighted by the multiplicity, and rows 3, 4
  // sum the absorbed multiplicities for the charge)
  __shared__ double s_tv2[2][kPushBlock];
  __shared__ unsigned int s_tn[5][kPushBlock];
  const int tx = threadIdx.x;
  s_tv2[0][tx] = s_tv2[1][tx] = 0.0;
  s_tn[0][tx] = s_tn[1][tx] = s_tn[2][tx] = s_tn[3][tx] = s_tn[4][tx] = 0u;
  const long long n = min((long long)a.cnt->n[a.cur_in][a.species], a.cap);
  const uint32_t step = a.cnt->step;
  if (blockIdx.x == 0 && threadIdx.x == 0)
    a.cnt->pushed[a.species] += (unsigned long long)n - a.cnt->n_tomb[a.species];
  const Grid& g = a.g;
  const float dt_f = (float)g.dt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* out_count = &a.cnt->n[a.cur_in ^ 1][a.species];
  using Particle = typename PTraits<S>::P;
  const long long round = (long long)kPushBlock * kIlp;
  for (long long base = (long long)blockIdx.x * round; base < n; base += (long long)gridDim.x * round) {
    Particle p[kIlp];
    bool valid[kIlp], keep[kIlp], ionize[kIlp];
    int cell_n[kIlp];
    int ch_ion[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const long long i = base + (long long)u * kPushBlock + threadIdx.x;
      valid[u] = i < n;
      keep[u] = ionize[u] = false;
      ch_ion[u] = -1;
      cell_n[u] = 0;
      if (valid[u]) p[u] = store_read(a.in, g, i);
    }
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      if (!valid[u]) continue;
      if (p[u].pid == kPidDead) continue;  // neutrals and ions converted in the last step are dropped here
      if (!PIC_BOUNDS(particle_cell(p[u]) >= 0 && particle_cell(p[u]) < g.ncell, a.cnt)) continue;
      cell_n[u] = (int)particle_cell(p[u]);
      if (CHARGED) {
        const auto e = p[u].gather(g, a);
        p[u].kick(a, e);
      }
      const int side = p[u].drift(g);  // -1 cathode, +1 anode, 0 inside
      if (side != 0) {
        const int b = side < 0 ? 0 : 1;
        s_tn[b][tx] += 1u;
        s_tn[3 + b][tx] += p[u].mw;
        s_tv2[b][tx] += (double)p[u].mw * p[u].v2();
        if (side < 0 && a.hits.n) {
          double xc, yc;
          p[u].cathode_point(g, xc, yc);
          const double3 v = p[u].vel();
          log_cathode_hit(a.hits, p[u].pid, a.species, step, xc, yc, v.x, v.y, v.z);
        }
        continue;
      }
      if (!PIC_BOUNDS(particle_cell(p[u]) >= 0 && particle_cell(p[u]) < g.ncell, a.cnt)) continue;
      keep[u] = true;
      if (MCC) {
        const float nb = mcc_nu_bound(a.mc, cell_n[u], a.mc.count_in_field ? p[u].nc : -1.f);
        if (nb <= 0.f) continue;
        const float cnt0 = a.mc.count_in_field ? p[u].nc : -1.f;
        const uint4 d = draw(a.mc.key, p[u].pid, step, TAG_MCC);
        const float v2f = p[u].v2f(), U32 = u01_32(d.x);
        if (!mcc_cannot_collide(nb, v2f, U32, dt_f)) {
          int ch = mcc_decide32(a.mc, cell_n[u], v2f, U32, dt_f, cnt0);
          if (ch == -2) ch = mcc_exact_dt(a.mc, cell_n[u], p[u].v2(), u01_64(d.x, d.y), g.dt);
          if (ch >= 0) {
            if (a.mc.ch[ch].kind == XS_ELASTIC) {
              p[u].scatter_isotropic(draw(a.mc.key, p[u].pid, step, TAG_SCATTER));
              s_tn[2][tx] += 1u;
            } else if (a.mc.bg_mode) {
              // fixed-background test mode: counted, nothing consumed or created
              atomicAdd(a.mc.ch[ch].kind == XS_CHARGE_EXCHANGE ? &a.cnt->n_cx : &a.cnt->n_ion, 1ull);
            } else {
              ionize[u] = true;
              ch_ion[u] = ch;
            }
          }
        }
      }
    }
    // block-wide slot reservation for the whole round
    unsigned ball[kIlp];
    unsigned wtot = 0;
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      ball[u] = __ballot_sync(0xffffffffu, keep[u]);
      wtot += __popc(ball[u]);
    }
    if (lane == 0) s_wcnt[warp] = wtot;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int tot = 0;
      for (int w = 0; w < kPushWarps; ++w) {
        const unsigned int c = s_wcnt[w];
        s_wcnt[w] = tot;
        tot += c;
      }
      s_base = tot ? atomicAdd(out_count, (unsigned long long)tot) : 0ull;
      // an overflowing round (ERR_CAPACITY below) caps the count again after its
      // own add, so the count ends at min(kept, capacity) and no later kernel
      // indexes past the store
      if (s_base + tot > (unsigned long long)a.cap) atomicMin(out_count, (unsigned long long)a.cap);
    }
    __syncthreads();
    unsigned long long wbase = s_base + s_wcnt[warp];
    __syncthreads();  // s_wcnt / s_base are rewritten in the next round
    bool stored[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const unsigned long long slot = wbase + __popc(ball[u] & ((1u << lane) - 1u));
      wbase += __popc(ball[u]);
      stored[u] = false;
      if (!keep[u]) continue;
      if (slot >= (unsigned long long)a.cap) {
        atomicOr(&a.cnt->error, ERR_CAPACITY);
        continue;
      }
      store_write_p(a.out, slot, p[u]);
      stored[u] = true;
      if (ionize[u]) {
        const unsigned int e = atomicAdd(&a.cnt->n_events, 1u);
        if (e < (unsigned int)a.ev_cap) {
          Event ev;
          ev.pid = p[u].pid;
          ev.cell = (uint32_t)cell_n[u];
          ev.slot = (uint32_t)slot;
          ev.ch = (int16_t)ch_ion[u];
          ev.kind = (int16_t)a.mc.ch[ch_ion[u]].kind;
          ev.E_eV = a.mc.half_m_over_e * p[u].v2();  // velocity unchanged since the decision
          ev.victim = -1;
          ev.next = atomicExch(&a.ev_head[cell_n[u]], (int)e);
          a.ev[e] = ev;
        } else {
          atomicOr(&a.cnt->error, ERR_EVENTS);
        }
      }
      if (NEUTRAL && a.ev_head != nullptr && a.ev_head[cell_n[u]] >= 0) {
        // candidate victim of an ionization or charge exchange in its cell at x^n
        const unsigned int c = atomicAdd(&a.cnt->n_cands, 1u);
        if (c < (unsigned int)a.cand_cap) {
          const uint4 k = draw(a.mc.key, p[u].pid, step, TAG_VICTIM);
          Cand cd;
          cd.key = ((unsigned long long)k.x << 32) | (unsigned long long)p[u].pid;
          cd.slot = (uint32_t)slot;
          cd.next = atomicExch(&a.cand_head[cell_n[u]], (int)c);
          a.cand[c] = cd;
          a.cand_cell[c] = (uint32_t)cell_n[u];
        } else {
          atomicOr(&a.cnt->error, ERR_EVENTS);
        }
      }
    }
    // a3 of the next step while the particles are at hand: charge (or neutral
    // count) at x^{n+1} of every particle kept
    if (a.nd.on) {
#pragma unroll
      for (int u = 0; u < kIlp; ++u) next_deposit<CHARGED, NEUTRAL>(a, p[u], stored[u]);
    }
  }
  // block totals of the tallies by warp 0: counts in integers, the FP64 sums of
  // v^2 only when the block absorbed something (FP64 is a narrow pipe on GB300)
  __syncthreads();
  if (warp == 0) {
    unsigned int n0 = 0, n1 = 0, nel = 0, m0 = 0, m1 = 0;
    for (int t = lane; t < kPushBlock; t += 32) {
      n0 += s_tn[0][t];
      n1 += s_tn[1][t];
      nel += s_tn[2][t];
      m0 += s_tn[3][t];
      m1 += s_tn[4][t];
    }
    n0 = __reduce_add_sync(0xffffffffu, n0);
    n1 = __reduce_add_sync(0xffffffffu, n1);
    nel = __reduce_add_sync(0xffffffffu, nel);
    m0 = __reduce_add_sync(0xffffffffu, m0);
    m1 = __reduce_add_sync(0xffffffffu, m1);
    if (n0 + n1 > 0) {
      double v0 = 0.0, v1 = 0.0;
      for (int t = lane; t < kPushBlock; t += 32) {
        v0 += s_tv2[0][t];
        v1 += s_tv2[1][t];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
      }
      if (lane == 0) {
        const int s = a.species;
        const double ke = 0.5 * a.mass * a.weight, qw = a.charge * a.weight;
        if (n0) {
          atomicAdd(&a.cnt->abs_cathode[s], (unsigned long long)n0);
          atomicAdd(&a.cnt->abs_energy_cathode[s], ke * v0);
          atomicAdd(&a.cnt->q_cathode_step, qw * (double)m0);
        }
        if (n1) {
          atomicAdd(&a.cnt->abs_anode[s], (unsigned long long)n1);
          atomicAdd(&a.cnt->abs_energy_anode[s], ke * v1);
          atomicAdd(&a.cnt->q_anode_step, qw * (double)m1);
        }
      }
    }
    if (lane == 0 && nel) atomicAdd(&a.cnt->n_el, (unsigned long long)nel);
  }
}

// ---------------------------------------------------------------------------
// a9: resolve of the events that need a victim (ionization, charge exchange)
// ---------------------------------------------------------------------------
// Rank of each event among the events of its cell by primary pid, then its
// victim: the rank-th smallest (key, pid) candidate of that cell, i.e. the
// candidate with exactly that many smaller keys. Keys are unique (they carry
// the pid), so the two searches below give the same victim.
// Few events and candidates (events x candidates <= kScanWork, the usual step):
// one block per event scans the flat candidate array (its eight warps take
// interleaved chunks, so the scan is a few rounds of coalesced loads, not a
// chain of dependent ones), gathers its cell's keys into shared memory and
// counts ranks there; a cell with more than kRankCand candidates falls back to
// the list walk. Otherwise one thread per event walks its cell's candidate list
// by repeated minimum selection (the flat scan would cost events x candidates).
constexpr int kRankCand = 256;
constexpr int kRankWarps = 8;
constexpr unsigned long long kScanWork = 1ull << 22;

__device__ int victim_by_list(const ResolveArgs& a, uint32_t cell, int r) {
  unsigned long long prev = 0;
  bool have_prev = false;
  int victim = -1;
  for (int s = 0; s <= r; ++s) {
    unsigned long long best = ~0ull;
    int bi = -1;
    int g2 = 0;
    for (int c = a.cand_head[cell]; c >= 0 && g2 < (1 << 22); c = a.cand[c].next, ++g2) {
      const unsigned long long k = a.cand[c].key;
      if ((!have_prev || k > prev) && k < best) {
        best = k;
        bi = c;
      }
    }
    if (bi < 0) return -1;
    prev = best;
    have_prev = true;
    victim = bi;
  }
  return victim;
}

__device__ __forceinline__ int event_rank(const ResolveArgs& a, uint32_t cell, uint32_t pid) {
  int r = 0;
  int guard = 0;
  for (int j = a.ev_head[cell]; j >= 0 && guard < (1 << 22); j = a.ev[j].next, ++guard)
    if (a.ev[j].pid < pid) ++r;
  return r;
}

__device__ __forceinline__ void finish_event(const ResolveArgs& a, long long e, uint32_t pid, int victim) {
  a.ev[e].victim = victim;
  // sort key for the apply order: successful ionizations by primary pid, then
  // successful charge exchanges by primary pid, then the suppressed events
  const bool cx = a.ev[e].kind == XS_CHARGE_EXCHANGE;
  a.sort_keys[e] = ((unsigned long long)(victim < 0 ? 1 : 0) << 33) | ((unsigned long long)(cx ? 1 : 0) << 32) | pid;
  a.sort_vals[e] = (uint32_t)e;
  if (victim >= 0) {
    atomicAdd(&a.cnt->n_success, 1u);
    if (cx) atomicAdd(&a.cnt->n_success_cx, 1u);
  }
}

__global__ void __launch_bounds__(kRankWarps * 32) k_resolve_rank(ResolveArgs a) {
  __shared__ unsigned long long sk[kRankCand];
  __shared__ int si[kRankCand];
  __shared__ int s_m, s_victim;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned int ne = min(a.cnt->n_events, (unsigned int)a.ev_cap);
  const unsigned int nc = min(a.cnt->n_cands, (unsigned int)a.cand_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt->ev_sort_n = ne;
  if ((unsigned long long)ne * nc > kScanWork) {
    for (long long e = gtid(); e < ne; e += gstride()) {
      const uint32_t cell = a.ev[e].cell, pid = a.ev[e].pid;
      finish_event(a, e, pid, victim_by_list(a, cell, event_rank(a, cell, pid)));
    }
    return;
  }
  const unsigned lt = (1u << lane) - 1u;
  // event e on block e mod G: tens of events, each scanned by a whole block
  for (long long e = blockIdx.x; e < ne; e += gridDim.x) {
    const uint32_t cell = a.ev[e].cell, pid = a.ev[e].pid;
    if (threadIdx.x == 0) {
      s_m = 0;
      s_victim = -1;
    }
    __syncthreads();
    // this cell's candidates: warp w takes chunks w, w + 8, ... of 256 (eight loads per lane in flight)
    for (unsigned base = (unsigned)w * 256u; base < nc; base += 256u * kRankWarps) {
      bool match[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const unsigned c = base + 32u * q + lane;
        match[q] = c < nc && a.cand_cell[c] == cell;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const unsigned bal = __ballot_sync(0xffffffffu, match[q]);
        if (!bal) continue;
        int at = 0;
        if (lane == 0) at = atomicAdd(&s_m, __popc(bal));
        at = __shfl_sync(0xffffffffu, at, 0);
        const int pos = at + __popc(bal & lt);
        if (match[q] && pos < kRankCand) {
          const unsigned c = base + 32u * q + lane;
          sk[pos] = a.cand[c].key;
          si[pos] = (int)c;
        }
      }
    }
    __syncthreads();
    const int m = s_m;
    if (m <= kRankCand) {
      const int r = event_rank(a, cell, pid);  // every thread the same
      for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const unsigned long long kq = sk[q];
        int below = 0;
        for (int t = 0; t < m; ++t) below += sk[t] < kq ? 1 : 0;
        if (below == r) s_victim = si[q];  // keys are unique: one thread at most
      }
    } else if (threadIdx.x == 0) {
      s_victim = victim_by_list(a, cell, event_rank(a, cell, pid));
    }
    __syncthreads();
    if (threadIdx.x == 0) finish_event(a, e, pid, s_victim);
    __syncthreads();  // s_m, s_victim, sk, si are reused by the next event
  }
}

// Counters of the resolved step: outcomes, the stores' new lengths, pids.
__device__ void resolve_commit(DevCounters* cnt, const ResolveCommit& c) {
  const unsigned int ne = min(cnt->n_events, (unsigned int)c.ev_cap);
  const unsigned int ns = cnt->n_success;
  const unsigned int ncx = cnt->n_success_cx;
  const unsigned int nion = ns - ncx;
  cnt->n_ion += nion;
  cnt->n_cx += ncx;
  cnt->n_supp += ne - ns;
  if (c.e_sp >= 0) {
    const unsigned long long a = cnt->n[c.e_out][c.e_sp] + nion;
    cnt->n[c.e_out][c.e_sp] = a > (unsigned long long)c.e_cap ? c.e_cap : a;
  }
  const unsigned long long b = cnt->n[c.i_out][c.i_sp] + ns;
  cnt->n[c.i_out][c.i_sp] = b > (unsigned long long)c.i_cap ? c.i_cap : b;
  const unsigned long long d = cnt->n[c.n_out][c.n_sp] + ncx;
  cnt->n[c.n_out][c.n_sp] = d > (unsigned long long)c.n_cap ? c.n_cap : d;
  // tombstones: every victim and exchanging ion, or with variable weights the
  // ones converted whole (the others only lost multiplicity)
  cnt->n_tomb[c.n_sp] = c.weighted ? cnt->n_kill_n : ns;
  cnt->n_tomb[c.i_sp] = c.weighted ? cnt->n_kill_i : ncx;
  cnt->n_kill_n = cnt->n_kill_i = 0u;
  cnt->next_pid += c.weighted ? 3u * ns : nion;
}

// Successful events in apply order: ionizations (rank r < nion) then charge
// exchanges. Every victim neutral becomes an ion (slot ni_out + r). An
// ionization scales its primary electron and appends a secondary (pid and
// slot from r, so secondaries take pids in increasing primary pid); an exchange
// turns its primary ion into a neutral (slot nn_out + r - nion) and takes back
// the charge the push deposited for it at x^{n+1}.
// Variable weights: an event moves ms = min(multiplicity of the primary, of the
// victim). The victim (or the exchanging ion) with more keeps the rest in its
// slot and the moved part is written with a pid of its own (victim's part
// pid0 + ns + 2r, exchanging ion's part pid0 + ns + 2r + 1); the secondary has
// multiplicity ms; a primary electron moving less than its multiplicity loses
// the ionization energy with probability ms / multiplicity (the second uniform
// of the ionization's second draw).
template <class S>
__global__ void k_resolve_apply(ApplyArgs<S> a) {
  const unsigned int ns = a.cnt->n_success;
  const unsigned int nion = ns - a.cnt->n_success_cx;
  const unsigned long long ne_out = a.e_species >= 0 ? a.cnt->n[a.e_out][a.e_species] : 0ull;
  const unsigned long long ni_out = a.cnt->n[a.i_out][a.i_species];
  const unsigned long long nn_out = a.cnt->n[a.n_out][a.n_species];
  const uint32_t pid0 = a.cnt->next_pid;
  // event r on block r mod G (as for injection: each event's FP64 kinematics
  // then run on their own SM's FP64 pipe instead of queueing on one)
  for (long long r = blockIdx.x + (long long)gridDim.x * threadIdx.x; r < ns;
       r += (long long)gridDim.x * blockDim.x) {
    if (!PIC_BOUNDS(a.sorted_vals[r] < (uint32_t)a.ev_cap, a.cnt)) continue;
    const Event ev = a.ev[a.sorted_vals[r]];
    if (!PIC_BOUNDS(ev.victim >= 0 && ev.victim < a.cand_cap &&
                        (long long)ev.slot < (ev.kind == XS_CHARGE_EXCHANGE ? a.i_cap : a.e_cap),
                    a.cnt))
      continue;
    const Cand cd = a.cand[ev.victim];
    if (!PIC_BOUNDS(cd.slot < (uint32_t)a.n_cap, a.cnt)) continue;
    // victim neutral -> ion (position x^{n+1}, velocity and pid kept)
    const auto vn = store_read(a.n_st, a.g, cd.slot);
    const bool is_cx = r >= nion;
    const uint32_t mp = a.commit.weighted ? (is_cx ? a.i_st.mw[ev.slot] : a.e_st.mw[ev.slot]) : 1u;
    const uint32_t ms = min(mp, vn.mw);
    auto vm = vn;  // the part that converts
    if (ms == vn.mw) {
      store_kill(a.n_st, cd.slot);
      if (a.commit.weighted) atomicAdd(&a.cnt->n_kill_n, 1u);
    } else {
      a.n_st.mw[cd.slot] = vn.mw - ms;
      vm.mw = ms;
      vm.pid = pid0 + ns + 2u * (uint32_t)r;
    }
    const unsigned long long is = ni_out + r;
    if (is < (unsigned long long)a.i_cap) {
      store_write_p(a.i_st, is, vm);
      if (a.nd.on) deposit_one(a.g, vm, a.nd.rho32, a.nd.rho64, a.nd.qw_h3[a.i_species]);
    } else {
      atomicOr(&a.cnt->error, ERR_CAPACITY);
    }
    if (a.nd.on) atomicSub(&a.nd.ncount[a.n_species][cell_now(a.g, vn)], (int)ms);
    if (is_cx) {
      // charge exchange: the primary ion continues as a neutral
      auto pi = store_read(a.i_st, a.g, ev.slot);
      if (ms == mp) {
        store_kill(a.i_st, ev.slot);
        if (a.commit.weighted) atomicAdd(&a.cnt->n_kill_i, 1u);
      } else {
        a.i_st.mw[ev.slot] = mp - ms;
        pi.mw = ms;
        pi.pid = pid0 + ns + 2u * (uint32_t)r + 1u;
      }
      const unsigned long long os = nn_out + (r - nion);
      if (os < (unsigned long long)a.n_cap) {
        store_write_p(a.n_st, os, pi);
        if (a.nd.on) {
          deposit_one(a.g, pi, a.nd.rho32, a.nd.rho64, -a.nd.qw_h3[a.i_species]);
          atomicAdd(&a.nd.ncount[a.n_species][cell_now(a.g, pi)], (int)ms);
        }
      } else {
        atomicOr(&a.cnt->error, ERR_CAPACITY);
      }
      continue;
    }
    const XsDev& X = a.ch[ev.ch];
    const uint4 g0 = draw(a.key, ev.pid, a.cnt->step, TAG_IONIZE, 0);
    const uint4 g1 = draw(a.key, ev.pid, a.cnt->step, TAG_IONIZE, 1);
    const double Eex = ev.E_eV - X.thr;
    const double Us = u01_64(g0.x, g0.y);
    const double E2 = Us * Eex;
    const double E1 = (1.0 - Us) * Eex;
    const double sc = sqrt(E1 / ev.E_eV);
    // primary: direction kept, energy (1-U) (E - thr)
    auto pr = store_read(a.e_st, a.g, ev.slot);
    if (ms == mp || u01_64(g1.z, g1.w) < (double)ms / (double)mp) {
      pr.scale_v(sc);
      store_write_v(a.e_st, ev.slot, pr);
    }
    // secondary at the primary's new position
    const double us = sqrt(2.0 * E2 * kQe / a.e_mass);
    const double ct = 2.0 * u01_64(g0.z, g0.w) - 1.0;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    const double ph = 2.0 * kPi * u01_64(g1.x, g1.y);
    const uint32_t spid = pid0 + (uint32_t)r;
    auto sec = pr;
    sec.set_v(us * st * cos(ph), us * st * sin(ph), us * ct);
    sec.pid = spid;
    sec.mw = ms;
    const unsigned long long es = ne_out + r;
    if (es < (unsigned long long)a.e_cap) {
      store_write_p(a.e_st, es, sec);
      if (a.nd.on) deposit_one(a.g, sec, a.nd.rho32, a.nd.rho64, a.nd.qw_h3[a.e_species]);
    } else {
      atomicOr(&a.cnt->error, ERR_CAPACITY);
    }
    if (a.log) {
      a.log[3 * r] = ev.pid;
      a.log[3 * r + 1] = vn.pid;
      a.log[3 * r + 2] = spid;
    }
  }
  // the per-cell list heads of this step's events (and so of its candidates) go
  // back to empty; nothing in this kernel reads them
  const unsigned int ne = min(a.cnt->n_events, (unsigned int)a.commit.ev_cap);
  for (long long e = gtid(); e < ne; e += gstride()) {
    const uint32_t c = a.ev[e].cell;
    a.ev_head[c] = -1;
    a.cand_head[c] = -1;
  }
  // the last block to finish commits the step's counts (every block has read them)
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.cnt->resolve_ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    resolve_commit(a.cnt, a.commit);
    a.cnt->resolve_ticket = 0u;
  }
}


// ---------------------------------------------------------------------------
// explicit instantiations through launchers
// ---------------------------------------------------------------------------
template <class S>
void launch_inject(const InjectArgs<S>& a, int grid, cudaStream_t st) {
  PIC_LAUNCH(grid, 256, 0, st, k_inject<S>)(a);
}

template <class S>
void launch_push(const PushArgs<S>& a, int role, bool mcc, int grid, cudaStream_t st) {
  if (role == ROLE_NEUTRAL)
    PIC_LAUNCH(grid, 256, 0, st, k_push<S, false, false, true>)(a);
  else if (mcc)
    PIC_LAUNCH(grid, 256, 0, st, k_push<S, true, true, false>)(a);
  else
    PIC_LAUNCH(grid, 256, 0, st, k_push<S, true, false, false>)(a);
}


void launch_resolve_rank(const ResolveArgs& a, int grid, cudaStream_t st) {
  PIC_LAUNCH(grid, kRankWarps * 32, 0, st, k_resolve_rank)(a);
}
template <class S>
void launch_resolve_apply(const ApplyArgs<S>& a, int grid, cudaStream_t st) {
  PIC_LAUNCH(grid, 256, 0, st, k_resolve_apply<S>)(a);
}

template void launch_inject<Store64>(const InjectArgs<Store64>&, int, cudaStream_t);
template void launch_inject<StoreMx>(const InjectArgs<StoreMx>&, int, cudaStream_t);
template void launch_push<Store64>(const PushArgs<Store64>&, int, bool, int, cudaStream_t);
template void launch_push<StoreMx>(const PushArgs<StoreMx>&, int, bool, int, cudaStream_t);
template void launch_resolve_apply<Store64>(const ApplyArgs<Store64>&, int, cudaStream_t);
template void launch_resolve_apply<StoreMx>(const ApplyArgs<StoreMx>&, int, cudaStream_t);

}  // namespace pic
