// spock_centre.cu -- the FP64 centre of the centred FP32 iteration.
//
// The centred iteration runs the SPOCK iteration (Alg. 4 with the operator T of
// the Chambolle-Pock step) on delta = v - c for an FP64 centre c, i.e. on the
// map D(delta) = T(c + delta) - c. prox_f is affine (Alg. 2 solves a linear
// system), so its part of D is the linear part applied to the increment plus
// the constant z+_c - z_c; L is linear; only the prox of g* is taken about the
// centre, in FP64. The kernels below build what one centre needs from T(c)
// and L z_c (both evaluated in FP64), and move the final increment into c.
#include <cuda_runtime.h>

#include "spock_problem.h"

namespace spock {

// cz = z+_c - z_c (FP32); per element e of eta, with a the translation of the
// element's set (the cost cones of Prop. 1; zero elsewhere):
//   A = (eta_c + alpha (L z_c))/alpha - a,  B = alpha (L z_c) - alpha a.
__global__ void k_centre(Prob<double> P, const double* __restrict__ c, const double* __restrict__ tc,
                         const double* __restrict__ lz, double alpha, float* __restrict__ cz,
                         double* __restrict__ A, double* __restrict__ B) {
  const long long nz = P.nz, ne = P.neta;
  const long long nq = (long long)(P.n - 1) * P.W;
  const int dN = P.nx + 2;
  const long long nqN = (long long)P.n_l * dN;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nz + ne;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < nz) {
      cz[i] = (float)(tc[i] - c[i]);
      continue;
    }
    const long long e = i - nz;
    double a = 0.0;
    if (e >= P.e_q && e < P.e_q + nq) {
      const long long r = e - P.e_q;
      const int j = (int)(r % P.W);
      a = P.acost ? P.acost[r] : (j == P.W - 2 ? 0.5 : (j == P.W - 1 ? -0.5 : 0.0));
    } else if (e >= P.e_qN && e < P.e_qN + nqN) {
      const long long r = e - P.e_qN;
      const int j = (int)(r % dN);
      a = P.acostN ? P.acostN[r] : (j == dN - 2 ? 0.5 : (j == dN - 1 ? -0.5 : 0.0));
    } else if (P.soft && e >= P.e_sf) {   // the soft costs' cones: (0, 1/2, -1/2)
      const int dS = P.nx + P.nu;
      const int j = (int)((e - P.e_sf) % (3 * dS + 2));
      a = (j == dS) ? 0.5 : (j == dS + 1 ? -0.5 : 0.0);
    }
    const double l = lz[e];
    A[e] = (c[nz + e] + alpha * l) / alpha - a;
    B[e] = alpha * l - alpha * a;
  }
}

// c += delta (the increment of the finished segment moves into the centre)
__global__ void k_centre_move(long long n, double* __restrict__ c, const float* __restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c[i] += (double)d[i];
}

// FP32 copy of the FP64 iterate
__global__ void k_centre_to_f32(long long n, const double* __restrict__ c, float* __restrict__ v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] = (float)c[i];
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 148 * 8) g = 148 * 8;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_centre(const Prob<double>& P, const double* c, const double* tc, const double* lz, double alpha,
                          float* cz, double* A, double* B, cudaStream_t st) {
  k_centre<<<grid_for(P.nz + P.neta), 256, 0, st>>>(P, c, tc, lz, alpha, cz, A, B);
  return cudaGetLastError();
}

cudaError_t launch_centre_move(long long n, double* c, const float* d, cudaStream_t st) {
  k_centre_move<<<grid_for(n), 256, 0, st>>>(n, c, d);
  return cudaGetLastError();
}

cudaError_t launch_centre_to_f32(long long n, const double* c, float* v, cudaStream_t st) {
  k_centre_to_f32<<<grid_for(n), 256, 0, st>>>(n, c, v);
  return cudaGetLastError();
}

}  // namespace spock
