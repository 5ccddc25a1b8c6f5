// pic_internal.cuh -- device-side types and helpers of the GB300 PIC/MCC library.
//
// Layout in HBM (per instance):
//   particle stores, two ping-pong buffers per species, structure of arrays:
//     FP64 path : x, y, z, vx, vy, vz (double) + pid (u32)            52 B/particle
//     MIXED path: cell (i32) + ox, oy, oz (f32, cell units in [0,1)) +
//                 vx, vy, vz (f32) + pid (u32)                           32 B/particle
//   grid: rho (nodes), phi (nodes), E at nodes (double4 / float4), neutral
//   counts (i32 per cell), solver vectors over the unknown nodes
//   (k = 1..nz-1) and the multigrid hierarchy.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

constexpr int kMaxSpecies = 8;
constexpr int kMaxXsec = 8;
constexpr int kMaxSources = 16;

// CODATA 2018 (SI)
constexpr double kQe = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kKB = 1.380649e-23;
constexpr double kPi = 3.14159265358979323846;

constexpr uint32_t kPidDead = 0xFFFFFFFFu;  // tombstone of a converted neutral or exchanged ion

// Philox counter layout (pid, step, tag, j); tags give each draw a purpose.
enum : uint32_t {
  TAG_MCC = 0,       // (U1): collision test and channel choice
  TAG_SCATTER = 1,   // (cos theta, phi) of an elastic scattering
  TAG_IONIZE = 2,    // j = 0: (energy split, cos theta), j = 1: (phi) of the secondary
  TAG_INJ_POS = 16,  // (radius, angle) on the emitter disk
  TAG_INJ_VXY = 17,  // Box-Muller pair -> vx, vy
  TAG_INJ_VZ = 18,   // Box-Muller (cos branch) -> |vz|
  TAG_INJ_Z = 19,    // fraction of the first partial step
  TAG_VICTIM = 32    // 32-bit ranking key of a neutral as ionization victim
};

enum : int { ROLE_ELECTRON = 0, ROLE_NEUTRAL = 1, ROLE_ION = 2 };
enum : int { XS_IONIZATION = 0, XS_ELASTIC = 1, XS_CHARGE_EXCHANGE = 2 };

// device error bits (DevCounters::error)
enum : int { ERR_CAPACITY = 1, ERR_EVENTS = 2, ERR_TIMEOUT = 4, ERR_NOCONV = 8, ERR_BOUNDS = 16 };

// Checked build (compiled with -DPIC_CHECKED, libpic_gb300_checked.so): every
// cell, slot and list index a particle kernel takes from memory is tested
// before use; a bad one records ERR_BOUNDS and the access is skipped. In the
// ordinary build the test is not compiled.
#ifdef PIC_CHECKED
#define PIC_BOUNDS(ok, cnt) ((ok) ? true : (atomicOr(&(cnt)->error, ERR_BOUNDS), false))
#else
#define PIC_BOUNDS(ok, cnt) true
#endif

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 draw(uint2 key, uint32_t pid, uint32_t step, uint32_t tag, uint32_t j = 0) {
  return philox(make_uint4(pid, step, tag, j), key);
}

// FP64 uniform (m + 1/2) 2^-52 with m the top 52 bits of (a, b): built as the
// double 1 + m 2^-52 in [1,2) from its bit pattern, then shifted; both steps exact.
__device__ __forceinline__ double u01_64(uint32_t a, uint32_t b) {
  const double one_m = __hiloint2double(0x3FF00000 | (a >> 12), (a << 20) | (b >> 12));
  return (one_m - 1.0) + 0x1p-53;
}
// FP32 companion of u01_64 from the same a: the top 23 bits as the float
// 1 + m 2^-23 in [1,2), shifted to the midpoint of its interval, so that
// |u01_32(a) - u01_64(a, b)| <= 2^-24 (no int->float conversion).
__device__ __forceinline__ float u01_32(uint32_t a) {
  return (__uint_as_float(0x3F800000u | (a >> 9)) - 1.0f) + 0x1p-24f;
}

// ---------------------------------------------------------------------------
// Division by a loop-invariant divisor without integer division (whose int <->
// float conversions run on GB300's narrow FP64/conversion pipe): for 1 < d < 2^31
// and 0 <= n < 2^31, n / d = umulhi(n, m) >> (s - 1) with s = ceil(log2 d),
// m = ceil(2^(31+s) / d) (Granlund-Montgomery round-up method).
// ---------------------------------------------------------------------------
struct FastDiv {
  uint32_t m;
  int s, d;
};
inline FastDiv make_fastdiv(int d) {
  FastDiv f{0u, 0, d};
  if (d > 1) {
    int s = 0;
    while ((1ll << s) < (long long)d) ++s;
    const unsigned __int128 num = (unsigned __int128)1 << (31 + s);
    f.m = (uint32_t)((num + (unsigned __int128)(d - 1)) / (unsigned __int128)d);
    f.s = s;
  }
  return f;
}
__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
  return f.d == 1 ? n : (int)(__umulhi((unsigned)n, f.m) >> (f.s - 1));
}
// n mod d for any int n (periodic wrap), d = f.d
__device__ __forceinline__ int fwrap(int n, const FastDiv& f) {
  if (n >= 0 && n < f.d) return n;
  if (n >= f.d) return n - fdiv(n, f) * f.d;
  const int a = -n - 1;  // n = -(a + 1)
  return f.d - 1 - (a - fdiv(a, f) * f.d);
}

// ---------------------------------------------------------------------------
// Grid description
// ---------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz;
  double h, inv_h, dt;
  double Lx, Ly, Lz, inv_Lx, inv_Ly;
  double phi_c, phi_a;
  float h_f, inv_h_f, dt_over_h_f;
  long long ncell, nnode, nplane;
  FastDiv fdx, fdy;  // division by nx and ny
};

__device__ __forceinline__ double wrap_coord(double x, double L, double invL) {
  double r = x - L * floor(x * invL);
  if (r >= L) r -= L;
  if (r < 0.0) r += L;
  return r;
}

// ---------------------------------------------------------------------------
// Particle stores
// ---------------------------------------------------------------------------
// mw: integer multiplicities (a particle stands for mw x the species weight)
// when the instance has variable weights, else nullptr (every particle 1)
struct Store64 {
  double *x, *y, *z, *vx, *vy, *vz;
  uint32_t* pid;
  uint32_t* mw;
};
struct StoreMx {
  int32_t* cell;
  float *ox, *oy, *oz, *vx, *vy, *vz;
  uint32_t* pid;
  uint32_t* mw;
};

// ---------------------------------------------------------------------------
// Cross-section channels
// ---------------------------------------------------------------------------
constexpr int kXsBuckets = 4096;

struct XsDev {
  int kind, projectile, target, product, n;
  double thr;
  float thr_f;
  const double* E;     // [n]
  const double* sig;   // [n]
  const float* Ef;     // [n]
  const float* sigf;   // [n]
  const float* slopef; // [n - 1] (sig[i+1] - sig[i]) / (E[i+1] - E[i]), rounded from FP64
  const int* bucket;   // [kXsBuckets] lowest candidate interval per log-bucket
  float lnE0, inv_dln; // bucket = (ln E - lnE0) * inv_dln
};

// ---------------------------------------------------------------------------
// Device counters of one instance (one allocation, zero-initialised)
// ---------------------------------------------------------------------------
struct DevCounters {
  unsigned long long n[2][kMaxSpecies];  // live slots (incl. tombstones) in buffer b
  unsigned long long injected[kMaxSpecies];
  unsigned long long abs_cathode[kMaxSpecies], abs_anode[kMaxSpecies];
  double abs_energy_cathode[kMaxSpecies], abs_energy_anode[kMaxSpecies];
  double q_cathode_step, q_anode_step;
  unsigned long long n_ion, n_el, n_supp, n_cx;
  unsigned long long n_tomb[kMaxSpecies];
  unsigned int n_events;      // events needing a victim this step (ionization, charge exchange)
  unsigned int n_success;     // of which found a victim
  unsigned int n_success_cx;  // of which charge exchanges
  unsigned int n_cands;    // victim candidates this step
  unsigned int next_pid;
  int error;
  int cg_iters;
  double cg_resid;
  unsigned long long ev_sort_n;  // events to order this step (min(n_events, capacity))
  unsigned long long pushed[kMaxSpecies];  // cumulative particle pushes (metric units)
  unsigned int step;                       // index of the step being taken (Philox counter word 1)
  double anode_V;                          // anode potential of the next solve (external circuit)
  unsigned int resolve_ticket;             // blocks of the resolve launch finished (0 between launches)
  unsigned int n_kill_n, n_kill_i;         // variable weights: victims and exchanging ions wholly converted this step
};

// External circuit (the serial RC circuit between the electrodes): a source V0
// charges the anode through R, the gap holds capacitance C, and the charge the
// anode collects in a step flows onto it. Applied once per step, after the push.
struct Circuit {
  int on;
  double R, C, V0, dt;
};

// Injection counts of the current step (a1), kept on the device so that a step
// can be recorded once and replayed: the carry accumulator of every source
// advances here exactly as the host formula does (acc += mu; n = floor(acc);
// acc -= n, all FP64).
struct InjectPlan {
  int nsrc;
  int species[kMaxSources];
  double mu[kMaxSources];   // expected macroparticles per step
  double acc[kMaxSources];  // carry
  unsigned int ticket;       // blocks of the injection launch finished (0 between launches)
};

// Host-side count of kernel launches issued by the library (all handles).
// g_launches: launch operations issued to the GPU (a kernel, or a whole graph);
// g_kernels: kernels those operations run (a graph adds the kernel nodes it was
// recorded with, each conditional body once).
int sm_count();  // multiprocessors of the current device
extern unsigned long long g_launches;
extern unsigned long long g_kernels;
inline void count_kernel() {
  ++g_launches;
  ++g_kernels;
}
inline void count_graph(unsigned long long kernels) {
  ++g_launches;
  g_kernels += kernels;
}
#define PIC_LAUNCH(grid, block, smem, stream, ...) (::pic::count_kernel()), __VA_ARGS__<<<grid, block, smem, stream>>>

// Ionization event (one per ionizing collision, before victim choice)
struct Event {
  uint32_t pid;      // primary pid (electron or ion)
  uint32_t cell;     // primary's cell at x^n
  uint32_t slot;     // primary's slot in its species' new buffer
  int16_t ch;        // channel slot among the primary species' channels
  int16_t kind;      // XS_IONIZATION | XS_CHARGE_EXCHANGE
  double E_eV;       // pre-collision energy
  int32_t next;      // next event in the same cell (linked list), -1 = end
  int32_t victim;    // victim candidate index, -1 = suppressed
};

struct Cand {
  unsigned long long key;  // (Philox victim key << 32) | pid
  uint32_t slot;           // slot in the new neutral buffer
  int32_t next;            // next candidate of the same cell, -1 = end
};

// Warp-aggregated slot reservation: every active lane with `want` gets a
// distinct slot from *counter; lanes keep warp order.
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long* counter, bool want) {
  const unsigned mask = __ballot_sync(__activemask(), want);
  if (!want) return 0;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & ((1u << lane) - 1u));
}

__device__ __forceinline__ unsigned int warp_reserve32(unsigned int* counter, bool want) {
  const unsigned mask = __ballot_sync(__activemask(), want);
  if (!want) return 0;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned int base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned int)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & ((1u << lane) - 1u));
}

// grid-stride helpers
__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

}  // namespace pic
