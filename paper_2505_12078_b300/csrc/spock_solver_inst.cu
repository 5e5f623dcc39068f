// spock_solver_inst.cu -- one instantiation of the solver kernel, selected by
// -DSPOCK_T (float | double) and -DSPOCK_CH (column chunks of the mat-vecs);
// compiled once per variant so the variants build in parallel.
#include "spock_solver_kernel.cuh"

#define SPOCK_CAT2(a, b) a##b
#define SPOCK_CAT(a, b) SPOCK_CAT2(a, b)

namespace spock {

cudaError_t SPOCK_CAT(launch_solve_, SPOCK_SUFFIX)(const Prob<SPOCK_T>& P,
                                                    const SolveBufs<SPOCK_T>& B,
                                                    const SolveOpts& o, int tw, int grid,
                                                    int threads, cudaStream_t s) {
  return launch_ch<SPOCK_T, SPOCK_CH>(P, B, o, tw, grid, threads, s);
}

int SPOCK_CAT(max_grid_, SPOCK_SUFFIX)(int tw, int threads, int pipe_bytes, size_t extra, int* out) {
  return max_grid_ch<SPOCK_T, SPOCK_CH>(tw, threads, pipe_bytes, extra, out);
}

size_t SPOCK_CAT(smem_bytes_, SPOCK_SUFFIX)(int tw, int threads, int pipe_bytes) {
  return Views<SPOCK_T, SPOCK_CH>::bytes(threads, tw, pipe_bytes);
}

#ifdef SPOCK_WITH_BATCH
cudaError_t SPOCK_CAT(launch_batch_, SPOCK_SUFFIX)(const Prob<SPOCK_T>* probs, const SolveBufs<SPOCK_T>* bufs,
                                                    const int* tws, const SolveOpts& o, const BatchPlan& plan,
                                                    long long* cycles, size_t smem, int grid, cudaStream_t s) {
  return launch_batch_ch<SPOCK_T, SPOCK_CH>(probs, bufs, tws, o, plan, cycles, smem, grid, s);
}
int SPOCK_CAT(batch_grid_, SPOCK_SUFFIX)(size_t smem, int* out) {
  return batch_grid_ch<SPOCK_T, SPOCK_CH>(smem, out);
}
cudaError_t SPOCK_CAT(launch_serve_, SPOCK_SUFFIX)(const Prob<SPOCK_T>* probs, const SolveBufs<SPOCK_T>* bufs,
                                                    const int* tws, const ServeMeta<SPOCK_T>* meta,
                                                    const SolveOpts& o, const ServeReq* ring, ServeRes* res, int cap,
                                                    ServeCtl* ctl, ServeDev* dev, unsigned long long idle_ns,
                                                    size_t smem, int grid, cudaStream_t s) {
  return launch_serve_ch<SPOCK_T, SPOCK_CH>(probs, bufs, tws, meta, o, ring, res, cap, ctl, dev, idle_ns, smem,
                                            grid, s);
}
int SPOCK_CAT(serve_grid_, SPOCK_SUFFIX)(size_t smem, int* out) {
  return serve_grid_ch<SPOCK_T, SPOCK_CH>(smem, out);
}
size_t SPOCK_CAT(views_bytes_, SPOCK_SUFFIX)(int tw, int pipe_bytes) {
  return Views<SPOCK_T, SPOCK_CH>::bytes(256, tw, pipe_bytes);
}
#endif

}  // namespace spock
