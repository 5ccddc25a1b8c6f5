// pic_solver.cuh -- multigrid-preconditioned CG for the scaled 7-point operator.
#pragma once

#include <vector>

#include <cuda_runtime.h>

namespace pic {

struct MgLevel {
  int nx, ny, nz;  // cells of the level; unknown nodes nx * ny * (nz - 1)
  long long nu;
};

struct CgScalars {
  double rz, pq, alpha, beta, rr, bb;
  int it;
  int pad;
};

struct SolveResult {
  int iters;
  double resid_rel;
  bool converged;
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
  cudaError_t init(const std::vector<MgLevel>& plan);
  void release();
  void vcycle(const T* rhs, T* z, cudaStream_t s);
};

template <class T>
struct Pcg {
  long long n = 0;
  T *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double* part = nullptr;
  CgScalars* sc = nullptr;
  CgScalars* host_sc = nullptr;
  Mg<T> mg;
  cudaError_t init(const std::vector<MgLevel>& plan);
  void release();
  double read_scalar(int which, cudaStream_t s);
  int iterate(T* x, double rr0, double tol_abs, int maxit, cudaStream_t s, double* rr_out);
};

struct Solver {
  int precision = 0;  // 0 FP64, 1 mixed
  long long n = 0;
  std::vector<MgLevel> plan;
  double* b = nullptr;  // right-hand side over the unknowns
  double* part = nullptr;
  CgScalars* sc = nullptr;
  CgScalars* host_sc = nullptr;
  double* r64 = nullptr;
  float* d32 = nullptr;
  double inner_rtol = 1e-4;
  Pcg<double> p64;
  Pcg<float> p32;
  cudaError_t init(int nx, int ny, int nz, int precision);
  void release();
  double reduce_host(int G, cudaStream_t s);
  SolveResult solve(double* x, double rtol, int maxit, cudaStream_t s);
};

}  // namespace pic
