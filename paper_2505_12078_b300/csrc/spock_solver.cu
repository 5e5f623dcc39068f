// spock_solver.cu -- picks the solver kernel variant (precision, mat-vec
// width) for a problem; the variants are compiled from spock_solver_inst.cu.
#include <cuda_runtime.h>

#include "spock_dev.cuh"
#include "spock_internal.h"

namespace spock {

#define SPOCK_DECL(T, SUF)                                                                   \
  cudaError_t launch_solve_##SUF(const Prob<T>&, const SolveBufs<T>&, const SolveOpts&, int, \
                                 int, int, cudaStream_t);                                    \
  int max_grid_##SUF(int, int, int, size_t, int*);                                                  \
  size_t smem_bytes_##SUF(int, int, int);
SPOCK_DECL(float, f1)
SPOCK_DECL(float, f2)
SPOCK_DECL(double, d2)
SPOCK_DECL(double, d4)

int solver_chunks(int precision, int width) {
  const int vec = precision == 64 ? 2 : 4;
  const int ch = (width + 32 * vec - 1) / (32 * vec);
  if (precision == 32) return ch <= 1 ? 1 : 2;
  return ch <= 2 ? 2 : 4;
}

template <>
cudaError_t launch_solve<float>(const Prob<float>& P, const SolveBufs<float>& B, const SolveOpts& o,
                                int tw, int grid, int threads, cudaStream_t s) {
  if (solver_chunks(32, P.nx + P.nu) == 1) return launch_solve_f1(P, B, o, tw, grid, threads, s);
  return launch_solve_f2(P, B, o, tw, grid, threads, s);
}
template <>
cudaError_t launch_solve<double>(const Prob<double>& P, const SolveBufs<double>& B, const SolveOpts& o,
                                 int tw, int grid, int threads, cudaStream_t s) {
  if (solver_chunks(64, P.nx + P.nu) == 2) return launch_solve_d2(P, B, o, tw, grid, threads, s);
  return launch_solve_d4(P, B, o, tw, grid, threads, s);
}

int solver_max_grid(int precision, int tw, int threads, int D, int pipe_bytes, size_t extra, int* grid_out) {
  const int ch = solver_chunks(precision, D);
  if (precision == 64) {
    return ch == 2 ? max_grid_d2(tw, threads, pipe_bytes, extra, grid_out)
                   : max_grid_d4(tw, threads, pipe_bytes, extra, grid_out);
  }
  return ch == 1 ? max_grid_f1(tw, threads, pipe_bytes, extra, grid_out)
                 : max_grid_f2(tw, threads, pipe_bytes, extra, grid_out);
}

size_t solver_smem_bytes(int precision, int tw, int threads, int D, int pipe_bytes) {
  const int ch = solver_chunks(precision, D);
  if (precision == 64)
    return ch == 2 ? smem_bytes_d2(tw, threads, pipe_bytes) : smem_bytes_d4(tw, threads, pipe_bytes);
  return ch == 1 ? smem_bytes_f1(tw, threads, pipe_bytes) : smem_bytes_f2(tw, threads, pipe_bytes);
}

}  // namespace spock
