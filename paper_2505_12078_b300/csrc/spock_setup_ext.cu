// spock_setup_ext.cu -- offline data (FP64) of the parts of the problem
// statement beyond diagonal weights and box/ball sets:
//
//  * full weights (Sec. 3.2): every Q^c, R^c, Q_N^j given as a symmetric
//    positive definite matrix. L applies a factor F with F'F = W (Sec. 4.4
//    writes W^{1/2}; any factor serves, C-7): the upper Cholesky factor, then
//    scaled as F S^{-1} by the diagonal scalings of Sec. 5.4. Both F and F'
//    are stored row-major so that L and L* read them with coalesced loads.
//  * linear cost terms (Prop. 1 with S = I): the epigraph of
//    z'Wz + w'z is {(z, t): (F z, t/2, t/2) - a in SOC} with
//    a = (-F^{-T} w / 2, -kappa/8 + 1/2, -kappa/8 - 1/2), kappa = ||F^{-T} w||^2.
//    The scalings leave a unchanged, so it is computed from the unscaled data.
//  * ||L|| when L's Gram matrix has full blocks: per non-leaf node the
//    (x^i, u^i) block G'G + blockdiag(sum_c F_Q^c'F_Q^c, sum_c F_R^c'F_R^c), per
//    leaf the x^j block G_N'G_N + F_N'F_N (G: every constraint row, scaled);
//    their largest eigenvalue by power iteration with a Rayleigh quotient, one
//    CTA per node. The other blocks keep their closed forms (k_norm_L).
#include <cuda_runtime.h>
#include <math.h>

#include "spock_dev.cuh"
#include "spock_internal.h"

namespace spock {

namespace {

// In place: W (m x m, row-major, symmetric) -> its upper Cholesky factor F
// (F'F = W), lower triangle zeroed. One CTA per matrix. A pivot that is not
// positive sets *err (the data is then not positive definite).
__global__ void k_chol_upper(int m, double* __restrict__ W, int* __restrict__ err) {
  double* F = W + (size_t)blockIdx.x * m * m;
  __shared__ double s_piv;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      const double d = F[(size_t)k * m + k];
      if (!(d > 0.0)) {
        atomicExch(err, 1);
        s_piv = 1.0;
      } else {
        s_piv = sqrt(d);
      }
      F[(size_t)k * m + k] = s_piv;
    }
    __syncthreads();
    for (int j = k + 1 + threadIdx.x; j < m; j += blockDim.x) F[(size_t)k * m + j] /= s_piv;
    __syncthreads();
    const int r = m - k - 1;   // trailing (i, j), k < i <= j < m
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = k + 1 + e / r, j = k + 1 + e % r;
      if (j >= i) F[(size_t)i * m + j] -= F[(size_t)k * m + i] * F[(size_t)k * m + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x)
    if (e / m > e % m) F[e] = 0.0;
}

// w = F^{-T} lin (forward substitution with the lower triangular F') for
// nblk blocks of size m; full: F upper (m x m per block), else F is the
// diagonal sqrt(Wd) given as Wd (m per block). kap[b] += ||w||^2.
__global__ void k_ftinv(int nblk, int m, int full, const double* __restrict__ F, const double* __restrict__ lin,
                        double* __restrict__ w, double* __restrict__ kap) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
    const double* Fb = F + (size_t)b * (full ? (size_t)m * m : (size_t)m);
    const double* lb = lin + (size_t)b * m;
    double* wb = w + (size_t)b * m;
    double k2 = 0.0;
    for (int i = 0; i < m; ++i) {
      double v;
      if (full) {
        double s = lb[i];
        for (int k = 0; k < i; ++k) s -= Fb[(size_t)k * m + i] * wb[k];
        v = s / Fb[(size_t)i * m + i];
      } else {
        v = lb[i] / sqrt(Fb[i]);
      }
      wb[i] = v;
      k2 += v * v;
    }
    kap[b] += k2;
  }
}

// translation vectors: a[b] = (-w_x/2, -w_u/2, -kappa/8 + 1/2, -kappa/8 - 1/2)
// with w_x [nblk mx] (or null), w_u [nblk mu] (or null, mu = 0)
__global__ void k_translation(int nblk, int mx, int mu, const double* __restrict__ wx,
                              const double* __restrict__ wu, const double* __restrict__ kap,
                              double* __restrict__ a) {
  const int W = mx + mu + 2;
  const long long tot = (long long)nblk * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / W;
    const int k = (int)(e % W);
    double v;
    if (k < mx) v = wx ? -0.5 * wx[b * mx + k] : 0.0;
    else if (k < mx + mu) v = wu ? -0.5 * wu[b * mu + (k - mx)] : 0.0;
    else v = -0.125 * kap[b] + (k == W - 2 ? 0.5 : -0.5);
    a[e] = v;
  }
}

// F~ = F diag(1/S) (columns), and its transpose: F [nblk m m] upper factors,
// S [m]; out Ft (row-major F~) and FtT (row-major F~')
__global__ void k_scale_factor(long long nblk, int m, const double* __restrict__ F, const double* __restrict__ S,
                               double* __restrict__ Ft, double* __restrict__ FtT) {
  const long long per = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nblk * per;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / per;
    const int r = (int)((e % per) / m), k = (int)(e % m);
    const double v = F[e] / S[k];
    Ft[e] = v;
    FtT[b * per + (long long)k * m + r] = v;
  }
}

// largest eigenvalue of the (x^i, u^i) block (non-leaf i) or x^j block (leaf
// j) of L'L by power iteration; one CTA per node, vectors in shared memory
// (d <= MAXD). atomicMax of the bit pattern (non-negative doubles order as
// integers).
__global__ void k_norm_L_blocks(Prob<double> P, int iters, double rtol, unsigned long long* __restrict__ out) {
  const int node = blockIdx.x;
  const int nx = P.nx, nu = P.nu;
  const bool leaf = node >= P.n_nl;
  const int d = leaf ? nx : nx + nu;
  __shared__ double v[MAXD], y[MAXD], t[MAXD];
  __shared__ double s_red[32];
  __shared__ double s_lam, s_nrm;
  __shared__ int s_done;
  for (int k = threadIdx.x; k < d; k += blockDim.x) v[k] = 1.0;
  if (threadIdx.x == 0) { s_lam = 0.0; s_done = 0; }
  __syncthreads();
  auto block_sum = [&](double x) -> double {
    x = warp_sum(x);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = x;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += s_red[w];
    __syncthreads();
    return r;
  };
  // normalise the start vector
  {
    double nn = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) nn += v[k] * v[k];
    nn = sqrt(block_sum(nn));
    for (int k = threadIdx.x; k < d; k += blockDim.x) v[k] /= nn;
    __syncthreads();
  }
  for (int it = 0; it < iters && !s_done; ++it) {
    for (int k = threadIdx.x; k < d; k += blockDim.x) y[k] = 0.0;
    __syncthreads();
    // y = Gram(v): cost factors
    if (!leaf) {
      for (int c = P.ch_off[node]; c < P.ch_off[node + 1]; ++c) {
        // x part: F_Q' (F_Q v_x), u part: F_R' (F_R v_u) (diagonal factors when not full)
        for (int e = threadIdx.x; e < nx + nu; e += blockDim.x) {
          double s = 0.0;
          if (e < nx) {
            if (P.full) { const double* F = P.FQ + (size_t)(c - 1) * nx * nx + (size_t)e * nx; for (int k = 0; k < nx; ++k) s += F[k] * v[k]; }
            else s = P.qh[(size_t)(c - 1) * nx + e] * v[e];
          } else {
            const int f = e - nx;
            if (P.full) { const double* F = P.FR + (size_t)(c - 1) * nu * nu + (size_t)f * nu; for (int k = 0; k < nu; ++k) s += F[k] * v[nx + k]; }
            else s = P.rh[(size_t)(c - 1) * nu + f] * v[e];
          }
          t[e] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nx + nu; k += blockDim.x) {
          double s = 0.0;
          if (k < nx) {
            if (P.full) { const double* F = P.FQT + (size_t)(c - 1) * nx * nx + (size_t)k * nx; for (int e = 0; e < nx; ++e) s += F[e] * t[e]; }
            else s = P.qh[(size_t)(c - 1) * nx + k] * t[k];
          } else {
            const int f = k - nx;
            if (P.full) { const double* F = P.FRT + (size_t)(c - 1) * nu * nu + (size_t)f * nu; for (int e = 0; e < nu; ++e) s += F[e] * t[nx + e]; }
            else s = P.rh[(size_t)(c - 1) * nu + f] * t[k];
          }
          y[k] += s;
        }
        __syncthreads();
      }
      // selection rows: x box gx^2, u box and ball gu^2 each; the l1 rows
      // lambda - z, lambda + z add 2 I (their cross terms with lambda cancel)
      const int nub = (P.nbu ? 1 : 0) + (P.has_ball ? 1 : 0);
      const double l1s = (P.l1 > 0) ? 2.0 : 0.0;
      for (int k = threadIdx.x; k < nx + nu; k += blockDim.x) {
        if (k < nx) { if (P.nbx) y[k] += P.gx[k] * P.gx[k] * v[k]; }
        else y[k] += nub * P.gu[k - nx] * P.gu[k - nx] * v[k];
        y[k] += l1s * v[k];
      }
      __syncthreads();
      // general rows: G' (G v)
      for (int r = threadIdx.x; r < P.n_g; r += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nx + nu; ++k) s += P.Gg[(size_t)r * (nx + nu) + k] * v[k];
        t[r] = s;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < nx + nu; k += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < P.n_g; ++r) s += P.GgT[(size_t)k * P.n_g + r] * t[r];
        y[k] += s;
      }
      __syncthreads();
    } else {
      const long long jj = node - P.n_nl;
      for (int e = threadIdx.x; e < nx; e += blockDim.x) {
        double s = 0.0;
        if (P.full) { const double* F = P.FN + (size_t)jj * nx * nx + (size_t)e * nx; for (int k = 0; k < nx; ++k) s += F[k] * v[k]; }
        else s = P.qNh[jj * nx + e] * v[e];
        t[e] = s;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < nx; k += blockDim.x) {
        double s = 0.0;
        if (P.full) { const double* F = P.FNT + (size_t)jj * nx * nx + (size_t)k * nx; for (int e = 0; e < nx; ++e) s += F[e] * t[e]; }
        else s = P.qNh[jj * nx + k] * t[k];
        if (P.nbx) s += P.gN[k] * P.gN[k] * v[k];
        y[k] = s;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < P.n_gN; r += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nx; ++k) s += P.GgN[(size_t)r * nx + k] * v[k];
        t[r] = s;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < nx; k += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < P.n_gN; ++r) s += P.GgNT[(size_t)k * P.n_gN + r] * t[r];
        y[k] += s;
      }
      __syncthreads();
    }
    // Rayleigh quotient v'y (v has unit norm) and the next v = y / ||y||
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) { a += v[k] * y[k]; b += y[k] * y[k]; }
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
      s_nrm = sqrt(b);
      if (fabs(a - s_lam) <= rtol * a || !(s_nrm > 0.0)) s_done = 1;
      s_lam = a;
    }
    __syncthreads();
    if (s_nrm > 0.0)
      for (int k = threadIdx.x; k < d; k += blockDim.x) v[k] = y[k] / s_nrm;
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s_lam));
}

inline int grid_of(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 148 * 16) b = 148 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_chol_upper(int nmat, int m, double* W, int* err, cudaStream_t s) {
  if (nmat <= 0) return cudaSuccess;
  k_chol_upper<<<nmat, 256, 0, s>>>(m, W, err);
  return cudaGetLastError();
}

cudaError_t launch_ftinv(int nblk, int m, int full, const double* F, const double* lin, double* w, double* kap,
                         cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  k_ftinv<<<grid_of(nblk, 128), 128, 0, s>>>(nblk, m, full, F, lin, w, kap);
  return cudaGetLastError();
}

cudaError_t launch_translation(int nblk, int mx, int mu, const double* wx, const double* wu, const double* kap,
                               double* a, cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  k_translation<<<grid_of((long long)nblk * (mx + mu + 2), 256), 256, 0, s>>>(nblk, mx, mu, wx, wu, kap, a);
  return cudaGetLastError();
}

cudaError_t launch_scale_factor(long long nblk, int m, const double* F, const double* S, double* Ft, double* FtT,
                                cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  k_scale_factor<<<grid_of(nblk * m * m, 256), 256, 0, s>>>(nblk, m, F, S, Ft, FtT);
  return cudaGetLastError();
}

cudaError_t launch_norm_L_blocks(const Prob<double>& P, unsigned long long* out, cudaStream_t s) {
  k_norm_L_blocks<<<P.n, 128, 0, s>>>(P, 20000, 1e-15, out);
  return cudaGetLastError();
}

}  // namespace spock
