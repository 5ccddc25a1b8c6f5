// pic_solver.cuh -- multigrid-preconditioned CG for the scaled 7-point operator,
// recorded once per instance as a CUDA graph with device-side stopping.
#pragma once

#include <vector>

#include <cuda_runtime.h>

namespace pic {

struct MgLevel {
  int nx, ny, nz;  // cells of the level; unknown nodes nx * ny * (nz - 1)
  long long nu;
};

// Solver scalars (device resident)
struct SolveCtl {
  double bb, tol2, rr_true, resid_rel;
  double rr, rz, pq, alpha, beta, tol_in2;
  int it_total, it_inner, outer, maxit, converged, more;
  unsigned ticket;  // blocks finished in the current grid-wide sum (0 between launches)
  int ax_valid;     // Solver::ax holds A x for the current x
  int stopped;      // the last residual ended the outer loop
  int spec_timeout; // a copy of the exact coarse solve did not arrive in time (sticky until reported)
};

struct SolveResult {
  int iters;
  double resid_rel;
  bool converged;
  bool timeout;  // SolveCtl::spec_timeout
};

std::vector<MgLevel> mg_plan(int nx, int ny, int nz);

template <class T>
struct Mg {
  std::vector<MgLevel> levels;
  std::vector<T*> e, b, r;
  T* Ainv = nullptr;
  bool rb_ok = false;
  bool coarse_dense = false;
  int coarse_sweeps = 16;
  int fuse_from = -1;    // levels fuse_from..end run in one thread-block cluster (FP32), -1: none
  size_t fuse_smem = 0;  // its dynamic shared memory per block
  bool split0 = false;   // finest level in the colour-split layout (FP32, red-black, two levels or more)
  // FP32: the first level below the finest that fast diagonalization solves
  // exactly (x, y at most 64 and multiples of 4, at most 128 unknown planes);
  // the V-cycle stops there. -1: none (the deeper levels as above)
  int spectral_at = -1;
  float* spec_mem = nullptr;  // its bases and eigenvalues
  size_t spec_smem_plane = 0, spec_smem_z = 0;
  cudaError_t init(const std::vector<MgLevel>& plan);
  void release();
  // part, ctl given: the last half sweep also forms the PCG product r.z (returns true then)
  bool vcycle(const T* rhs, T* z, cudaStream_t s, double* part = nullptr, SolveCtl* ctl = nullptr);
};

template <class T>
struct Pcg {
  long long n = 0;
  T *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *d = nullptr;
  Mg<T> mg;
  cudaError_t init(const std::vector<MgLevel>& plan);
  void release();
};

// Solve of A x = b on the unknown nodes. FP64 path: outer loop of FP64 true
// residuals around an FP64 PCG on the correction (plain restarted PCG).
// Mixed path: the same loop is iterative refinement, the correction solved by
// an FP32 PCG to inner_rtol relative to the current residual.
struct Solver {
  int precision = 0;  // 0 FP64, 1 mixed
  long long n = 0;
  std::vector<MgLevel> plan;
  // FP64 path
  double* b = nullptr;   // right-hand side over the unknowns
  double* ax = nullptr;  // A x of the last FP64 residual (reused while x is unchanged)
  // MIXED path: phi = vac + hi + lo over the unknowns (hi = the phi32 view)
  float* f32 = nullptr;  // FP32 charge term h^2 rho / eps0 (no folded boundary terms)
  float* lo32 = nullptr;
  double* part = nullptr;
  SolveCtl* ctl = nullptr;
  SolveCtl* host_ctl = nullptr;
  double inner_rtol = 1e-6;
  int max_outer = 40;
  Pcg<double> p64;
  Pcg<float> p32;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long graph_kernels = 0;  // kernel nodes in graph (loop bodies once)
  cudaStream_t aux[2] = {nullptr, nullptr};  // capture streams of the two loop bodies
  cudaError_t init(int nx, int ny, int nz, int precision);
  void release();
  cudaError_t build_graph(double* x, float* phi32, double phi_c, double phi_a, int nz, double rtol, int maxit);
  cudaError_t build_graph_once(double* x, float* phi32, double phi_c, double phi_a, int nz, double rtol, int maxit);
  cudaError_t launch(cudaStream_t s);
  cudaError_t record(cudaStream_t s0);
  cudaError_t run_host(cudaStream_t s);
  cudaError_t invalidate(cudaStream_t s);
  // MIXED path: FP64 phi (unknown view, hx) from (hi, lo), and back (x = nullptr: phi = 0)
  cudaError_t phi64_from_ff(cudaStream_t s);
  cudaError_t ff_from_phi64(const double* x, cudaStream_t s);
  // arguments of the recorded solve (also used by the host-driven loop)
  double* hx = nullptr;
  float* hphi32 = nullptr;  // hi of the MIXED path (unknown view of phi32)
  double h_phi_a = 0.0;
  double h_phi_c = 0.0, h_dphi_dk = 0.0, h_rtol = 1e-8;
  int h_maxit = 1;
  // Dirichlet values folded into b on the first and last unknown planes
  float fold_first() const { return (float)(h_phi_c + (plan[0].nz == 2 ? h_phi_a : 0.0)); }
  float fold_last() const { return plan[0].nz == 2 ? 0.f : (float)h_phi_a; }
  SolveResult result(cudaStream_t s);
  // the same in two parts: enqueue the copy of the decision block, then (after
  // the caller synchronized the stream) read it
  cudaError_t result_async(cudaStream_t s);
  SolveResult result_read() const;
};

}  // namespace pic
