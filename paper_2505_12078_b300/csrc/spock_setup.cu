// spock_setup.cu -- offline part of SPOCK on the GPU (FP64) and the L / L*
// operator kernels.
//
//  * scale_dyn:   A~ = S_c A S_anc^{-1}, B~ = S_c B Su^{-1}, c~ = S_c c (Sec. 5.4)
//  * alg1_stage:  Alg. 1 for all nodes of one stage (one CTA per node):
//                 R~ = I + sum B'PB, Cholesky, K = -R~^{-1} sum B'PA,
//                 Abar = A + BK, P = I + K'K + sum Abar'P Abar
//  * build_*:     per-iteration factor matrices (see spock_dev.cuh)
//  * norm_L:      ||L|| from the block structure of L (Sec. 4.4): with diagonal
//                 Q, R and selection constraints, L splits into blocks per
//                 node whose Gram matrices are diagonal except the (y^i, s^i)
//                 block [I 0; -b' 1], whose largest squared singular value is
//                 1 + beta/2 + sqrt(beta + beta^2/4), beta = ||b^i||^2.
//  * apply_L / apply_Lt: eta = L z, z = L* eta (Sec. 4.4), any precision.
#include <cuda_runtime.h>
#include <math.h>

#include "spock_dev.cuh"
#include "spock_internal.h"

namespace spock {

// ---------------------------------------------------------------------------
__global__ void k_scale_dyn(int n, int n_nl, int nx, int nu, const int* __restrict__ anc,
                            const double* __restrict__ Sx, const double* __restrict__ SxN,
                            const double* __restrict__ Su, const double* __restrict__ A,
                            const double* __restrict__ B, const double* __restrict__ c,
                            double* __restrict__ At, double* __restrict__ Bt,
                            double* __restrict__ ct) {
  const long long nA = (long long)(n - 1) * nx * nx;
  const long long nB = (long long)(n - 1) * nx * nu;
  const long long nc = (long long)(n - 1) * nx;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nA + nB + nc;
       e += stride) {
    if (e < nA) {
      const long long node = e / (nx * nx);
      const int r = (int)((e / nx) % nx), k = (int)(e % nx);
      const int ch = (int)node + 1;
      const double sr = (ch >= n_nl) ? SxN[r] : Sx[r];
      const double sk = (anc[ch] >= n_nl) ? SxN[k] : Sx[k];
      At[e] = sr * A[e] / sk;
    } else if (e < nA + nB) {
      const long long f = e - nA;
      const long long node = f / (nx * nu);
      const int r = (int)((f / nu) % nx), k = (int)(f % nu);
      const int ch = (int)node + 1;
      const double sr = (ch >= n_nl) ? SxN[r] : Sx[r];
      Bt[f] = sr * B[f] / Su[k];
    } else {
      const long long f = e - nA - nB;
      const long long node = f / nx;
      const int r = (int)(f % nx);
      const int ch = (int)node + 1;
      const double sr = (ch >= n_nl) ? SxN[r] : Sx[r];
      ct[f] = c ? sr * c[f] : 0.0;
    }
  }
}

// P of the leaves = I
__global__ void k_leaf_P(int n, int n_nl, int nx, double* __restrict__ P) {
  const long long tot = (long long)(n - n_nl) * nx * nx;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)((e / nx) % nx), k = (int)(e % nx);
    P[(long long)n_nl * nx * nx + e] = (r == k) ? 1.0 : 0.0;
  }
}

// Alg. 1 for the parents p0 .. p0 + gridDim.x - 1 (one stage). Scratch per
// parent: Rt, L, Linv, Rinv (nu x nu), KA (nu x nx); per child: BtP (nu x nx),
// PAb (nx x nx).
__global__ void k_alg1_stage(int p0, int nx, int nu, const int* __restrict__ ch_off,
                             const double* __restrict__ At, const double* __restrict__ Bt,
                             double* __restrict__ P, double* __restrict__ K,
                             double* __restrict__ Rt, double* __restrict__ Lc,
                             double* __restrict__ Linv, double* __restrict__ Rinv,
                             double* __restrict__ KA, double* __restrict__ BtP,
                             double* __restrict__ PAb, double* __restrict__ Abar,
                             int* __restrict__ err) {
  const int i = p0 + blockIdx.x;
  const int c0 = ch_off[i], c1 = ch_off[i + 1];
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long nu2 = (long long)nu * nu, nunx = (long long)nu * nx, nx2 = (long long)nx * nx;
  double* R = Rt + i * nu2;
  double* L = Lc + i * nu2;
  double* Li = Linv + i * nu2;
  double* Ri = Rinv + i * nu2;
  double* KAi = KA + i * nunx;
  double* Ki = K + i * nunx;
  // 1. B~'P per child
  for (int c = c0; c < c1; ++c) {
    const double* Bc = Bt + (long long)(c - 1) * nx * nu;
    const double* Pc = P + (long long)c * nx2;
    double* BP = BtP + (long long)c * nunx;
    for (long long e = tid; e < nunx; e += nth) {
      const int r = (int)(e / nx), k = (int)(e % nx);
      double s = 0.0;
      for (int l = 0; l < nx; ++l) s += Bc[(long long)l * nu + r] * Pc[(long long)l * nx + k];
      BP[e] = s;
    }
  }
  __syncthreads();
  // 2. R~ = I + sum B'PB ; KA = sum B'PA
  for (long long e = tid; e < nu2; e += nth) {
    const int r = (int)(e / nu), s_ = (int)(e % nu);
    double s = (r == s_) ? 1.0 : 0.0;
    for (int c = c0; c < c1; ++c) {
      const double* Bc = Bt + (long long)(c - 1) * nx * nu;
      const double* BP = BtP + (long long)c * nunx;
      for (int l = 0; l < nx; ++l) s += BP[(long long)r * nx + l] * Bc[(long long)l * nu + s_];
    }
    R[e] = s;
  }
  for (long long e = tid; e < nunx; e += nth) {
    const int r = (int)(e / nx), k = (int)(e % nx);
    double s = 0.0;
    for (int c = c0; c < c1; ++c) {
      const double* Ac = At + (long long)(c - 1) * nx2;
      const double* BP = BtP + (long long)c * nunx;
      for (int l = 0; l < nx; ++l) s += BP[(long long)r * nx + l] * Ac[(long long)l * nx + k];
    }
    KAi[e] = s;
  }
  __syncthreads();
  // 3. Cholesky R~ = L L'
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  for (long long e = tid; e < nu2; e += nth) L[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < nu; ++j) {
    if (tid == 0) {
      double d = R[(long long)j * nu + j];
      for (int k = 0; k < j; ++k) d -= L[(long long)j * nu + k] * L[(long long)j * nu + k];
      if (!(d > 0.0)) { s_bad = 1; d = 1.0; }
      L[(long long)j * nu + j] = sqrt(d);
    }
    __syncthreads();
    const double djj = L[(long long)j * nu + j];
    for (int r = j + 1 + tid; r < nu; r += nth) {
      double s = R[(long long)r * nu + j];
      for (int k = 0; k < j; ++k) s -= L[(long long)r * nu + k] * L[(long long)j * nu + k];
      L[(long long)r * nu + j] = s / djj;
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicExch(err, 1);
  // 4. L^{-1} (lower), one column per thread
  for (int j = tid; j < nu; j += nth) {
    for (int r = 0; r < nu; ++r) Li[(long long)r * nu + j] = 0.0;
    Li[(long long)j * nu + j] = 1.0 / L[(long long)j * nu + j];
    for (int r = j + 1; r < nu; ++r) {
      double s = 0.0;
      for (int k = j; k < r; ++k) s += L[(long long)r * nu + k] * Li[(long long)k * nu + j];
      Li[(long long)r * nu + j] = -s / L[(long long)r * nu + r];
    }
  }
  __syncthreads();
  // 5. R~^{-1} = Linv' Linv
  for (long long e = tid; e < nu2; e += nth) {
    const int r = (int)(e / nu), s_ = (int)(e % nu);
    double s = 0.0;
    for (int k = max(r, s_); k < nu; ++k) s += Li[(long long)k * nu + r] * Li[(long long)k * nu + s_];
    Ri[e] = s;
  }
  __syncthreads();
  // 6. K = -R~^{-1} KA
  for (long long e = tid; e < nunx; e += nth) {
    const int r = (int)(e / nx), k = (int)(e % nx);
    double s = 0.0;
    for (int l = 0; l < nu; ++l) s += Ri[(long long)r * nu + l] * KAi[(long long)l * nx + k];
    Ki[e] = -s;
  }
  __syncthreads();
  // 7. Abar_c = A~_c + B~_c K ; PAb_c = P_c Abar_c
  for (int c = c0; c < c1; ++c) {
    const double* Ac = At + (long long)(c - 1) * nx2;
    const double* Bc = Bt + (long long)(c - 1) * nx * nu;
    double* Ab = Abar + (long long)(c - 1) * nx2;
    for (long long e = tid; e < nx2; e += nth) {
      const int r = (int)(e / nx), k = (int)(e % nx);
      double s = Ac[e];
      for (int l = 0; l < nu; ++l) s += Bc[(long long)r * nu + l] * Ki[(long long)l * nx + k];
      Ab[e] = s;
    }
  }
  __syncthreads();
  for (int c = c0; c < c1; ++c) {
    const double* Pc = P + (long long)c * nx2;
    const double* Ab = Abar + (long long)(c - 1) * nx2;
    double* PA = PAb + (long long)c * nx2;
    for (long long e = tid; e < nx2; e += nth) {
      const int r = (int)(e / nx), k = (int)(e % nx);
      double s = 0.0;
      for (int l = 0; l < nx; ++l) s += Pc[(long long)r * nx + l] * Ab[(long long)l * nx + k];
      PA[e] = s;
    }
  }
  __syncthreads();
  // 8. P_i = I + K'K + sum Abar' P Abar
  double* Pi = P + (long long)i * nx2;
  for (long long e = tid; e < nx2; e += nth) {
    const int r = (int)(e / nx), k = (int)(e % nx);
    double s = (r == k) ? 1.0 : 0.0;
    for (int l = 0; l < nu; ++l) s += Ki[(long long)l * nx + r] * Ki[(long long)l * nx + k];
    for (int c = c0; c < c1; ++c) {
      const double* Ab = Abar + (long long)(c - 1) * nx2;
      const double* PA = PAb + (long long)c * nx2;
      for (int l = 0; l < nx; ++l) s += Ab[(long long)l * nx + r] * PA[(long long)l * nx + k];
    }
    Pi[e] = s;
  }
}

// ---------------------------------------------------------------------------
// factor matrices of the iteration (FP64)
// ---------------------------------------------------------------------------
__global__ void k_build_MB(int n, int nx, int nu, int ld, const int* __restrict__ anc,
                           const double* __restrict__ Abar, const double* __restrict__ Bt,
                           const double* __restrict__ Rinv, double* __restrict__ MB) {
  const long long per = (long long)nx * ld;
  const long long tot = (long long)(n - 1) * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long cm1 = e / per;
    const int k = (int)((e % per) / ld), j = (int)(e % ld);
    double v = 0.0;
    if (j < nx) {
      v = Abar[cm1 * nx * nx + (long long)k * nx + j];
    } else if (j < nx + nu) {
      const int jj = j - nx;
      const int a = anc[cm1 + 1];
      const double* Bc = Bt + cm1 * nx * nu + (long long)k * nu;
      const double* Ri = Rinv + (long long)a * nu * nu;
      for (int l = 0; l < nu; ++l) v += Bc[l] * Ri[(long long)l * nu + jj];
    }
    MB[e] = v;
  }
}

__global__ void k_build_MF(int n, int nx, int nu, int ld, const double* __restrict__ Abar,
                           const double* __restrict__ Bt, double* __restrict__ MF) {
  const long long per = (long long)(nx + nu) * ld;
  const long long tot = (long long)(n - 1) * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long cm1 = e / per;
    const int k = (int)((e % per) / ld), j = (int)(e % ld);
    double v = 0.0;
    if (j < nx) {
      if (k < nx) v = Abar[cm1 * nx * nx + (long long)j * nx + k];
      else v = Bt[cm1 * nx * nu + (long long)j * nu + (k - nx)];
    }
    MF[e] = v;
  }
}

__global__ void k_build_MP_KT(int n_nl, int nx, int nu, int ldP, int ldK,
                              const double* __restrict__ K, const double* __restrict__ Rinv,
                              double* __restrict__ MP, double* __restrict__ KT) {
  const long long perP = (long long)nu * ldP, perK = (long long)nx * ldK;
  const long long totP = (long long)n_nl * perP, totK = (long long)n_nl * perK;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < totP + totK;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < totP) {
      const long long i = e / perP;
      const int k = (int)((e % perP) / ldP), j = (int)(e % ldP);
      double v = 0.0;
      if (j < nx) v = K[i * nu * nx + (long long)k * nx + j];
      else if (j < nx + nu) v = Rinv[i * nu * nu + (long long)k * nu + (j - nx)];
      MP[e] = v;
    } else {
      const long long f = e - totP;
      const long long i = f / perK;
      const int k = (int)((f % perK) / ldK), j = (int)(f % ldK);
      KT[f] = (j < nu) ? K[i * nu * nx + (long long)j * nx + k] : 0.0;
    }
  }
}

__global__ void k_build_Pc(int n, int nx, const double* __restrict__ P,
                           const double* __restrict__ ct, double* __restrict__ Pc) {
  const long long tot = (long long)(n - 1) * nx;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long cm1 = e / nx;
    const int r = (int)(e % nx);
    const double* Pm = P + (cm1 + 1) * nx * nx + (long long)r * nx;
    const double* cv = ct + cm1 * nx;
    double s = 0.0;
    for (int l = 0; l < nx; ++l) s += Pm[l] * cv[l];
    Pc[e] = s;
  }
}

// kc_i = sum_c MB_c' (P_c c_c): the part of the backward recursion of Alg. 2
// that does not depend on the iterate (zero when every c = 0)
__global__ void k_build_kc(int n_nl, int nx, int nu, int ld, const int* __restrict__ ch_off,
                           const double* __restrict__ MB, const double* __restrict__ Pc,
                           double* __restrict__ kc) {
  const int w = nx + nu;
  const long long tot = (long long)n_nl * w;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / w;
    const int j = (int)(e % w);
    double s = 0.0;
    for (int c = ch_off[i]; c < ch_off[i + 1]; ++c) {
      const double* M = MB + (long long)(c - 1) * nx * ld;
      const double* p = Pc + (long long)(c - 1) * nx;
      for (int k = 0; k < nx; ++k) s += M[(long long)k * ld + j] * p[k];
    }
    kc[e] = s;
  }
}

// cost square roots, constraint coefficients and scaled sets (Sec. 5.4)
__global__ void k_cost_con(int n, int n_nl, int nx, int nu, int nbx, int nbu, int has_ball,
                           const int* __restrict__ anc, const double* __restrict__ Sx,
                           const double* __restrict__ SxN, const double* __restrict__ Su,
                           double a_con, double a_conN, const double* __restrict__ Qd,
                           const double* __restrict__ Rd, const double* __restrict__ QNd,
                           const double* __restrict__ xlo, const double* __restrict__ xhi,
                           const double* __restrict__ ulo, const double* __restrict__ uhi,
                           const double* __restrict__ uball, double* __restrict__ qh,
                           double* __restrict__ rh, double* __restrict__ qNh,
                           double* __restrict__ gx, double* __restrict__ gu,
                           double* __restrict__ gN, double* __restrict__ box_lo,
                           double* __restrict__ box_hi, double* __restrict__ boxN_lo,
                           double* __restrict__ boxN_hi, double* __restrict__ ball) {
  const int n_l = n - n_nl;
  const int nbox = nbx + nbu;
  const long long s1 = (long long)(n - 1) * nx, s2 = s1 + (long long)(n - 1) * nu,
                  s3 = s2 + (long long)n_l * nx, s4 = s3 + nx + nu + nx,
                  s5 = s4 + (long long)n_nl * nbox, s6 = s5 + (long long)n_l * nx,
                  s7 = s6 + n_nl;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < s7;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < s1) {
      const long long cm1 = e / nx;
      const int k = (int)(e % nx);
      const int a = anc[cm1 + 1];
      const double S = (a >= n_nl) ? SxN[k] : Sx[k];
      qh[e] = sqrt(Qd[e]) / S;
    } else if (e < s2) {
      const long long f = e - s1;
      rh[f] = sqrt(Rd[f]) / Su[f % nu];
    } else if (e < s3) {
      const long long f = e - s2;
      qNh[f] = sqrt(QNd[f]) / SxN[f % nx];
    } else if (e < s4) {
      const int f = (int)(e - s3);
      if (f < nx) gx[f] = 1.0 / (Sx[f] * a_con);
      else if (f < nx + nu) gu[f - nx] = 1.0 / (Su[f - nx] * a_con);
      else gN[f - nx - nu] = 1.0 / (SxN[f - nx - nu] * a_conN);
    } else if (e < s5) {
      const long long f = e - s4;
      const long long i = f / nbox;
      const int r = (int)(f % nbox);
      if (r < nbx) {
        box_lo[f] = xlo[i * nx + r] / a_con;
        box_hi[f] = xhi[i * nx + r] / a_con;
      } else {
        box_lo[f] = ulo[i * nu + (r - nbx)] / a_con;
        box_hi[f] = uhi[i * nu + (r - nbx)] / a_con;
      }
    } else if (e < s6) {
      const long long f = e - s5;
      if (nbx) {
        boxN_lo[f] = xlo[(long long)n_nl * nx + f] / a_conN;
        boxN_hi[f] = xhi[(long long)n_nl * nx + f] / a_conN;
      }
    } else {
      const long long i = e - s6;
      if (has_ball) ball[i] = uball[i] / a_con;
    }
  }
}

// With soft-constraint costs, component k of (x^i, u^i) pairs with theta^i_k:
// L'L on (z_k, theta_k) is [g + 1, -1; -1, w^2 + 2] (the row theta - z adds 1
// and -1, theta >= 0 adds 1, the soft cone w^2): its largest eigenvalue.
__device__ __forceinline__ double soft_pair(double g, double w) {
  const double a = g + 1.0, b = w * w + 2.0;
  return 0.5 * (a + b) + sqrt(0.25 * (a - b) * (a - b) + 1.0);
}

// ||L||^2 as the max over the diagonal-Gram blocks of L (see file header)
__global__ void k_norm_L(int n, int n_nl, int nx, int nu, int nbx, int nub, double xu_shift, int ys_block,
                         const double* __restrict__ soft_w,
                         const int* __restrict__ ch_off, const double* __restrict__ prob,
                         const double* __restrict__ qh, const double* __restrict__ rh,
                         const double* __restrict__ qNh, const double* __restrict__ gx,
                         const double* __restrict__ gu, const double* __restrict__ gN,
                         unsigned long long* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double lam = 0.5;   // tau^c (non-leaf blocks) or s^j (leaf blocks): 1/4 + 1/4
    if (i < n_nl) {
      const int c0 = ch_off[i], c1 = ch_off[i + 1];
      for (int k = 0; k < nx; ++k) {
        double s = (nbx ? gx[k] * gx[k] : 0.0) + xu_shift;
        for (int c = c0; c < c1; ++c) s += qh[(long long)(c - 1) * nx + k] * qh[(long long)(c - 1) * nx + k];
        lam = fmax(lam, soft_w ? soft_pair(s, soft_w[k]) : s);
      }
      for (int k = 0; k < nu; ++k) {
        double s = nub * gu[k] * gu[k] + xu_shift;
        for (int c = c0; c < c1; ++c) s += rh[(long long)(c - 1) * nu + k] * rh[(long long)(c - 1) * nu + k];
        lam = fmax(lam, soft_w ? soft_pair(s, soft_w[nx + k]) : s);
      }
      if (ys_block) {   // AV@R's (y, s) block, beta = ||b||^2 (other risks: on the host)
        double beta = 1.0;
        for (int c = c0; c < c1; ++c) beta += prob[c] * prob[c];
        lam = fmax(lam, 1.0 + 0.5 * beta + sqrt(beta + 0.25 * beta * beta));
      }
    } else {
      const int j = i - n_nl;
      for (int k = 0; k < nx; ++k) {
        double s = (nbx ? gN[k] * gN[k] : 0.0) + qNh[(long long)j * nx + k] * qNh[(long long)j * nx + k];
        lam = fmax(lam, s);
      }
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(lam));
  }
}

template <class Src, class Dst>
__global__ void k_convert(long long n, const Src* __restrict__ a, Dst* __restrict__ b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    b[e] = (Dst)a[e];
}

// ---------------------------------------------------------------------------
// eta = L z (Sec. 4.4)
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_apply_L(Prob<T> P, const int* __restrict__ ynode, const T* __restrict__ z,
                          T* __restrict__ eta) {
  const int nx = P.nx, nu = P.nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < P.neta;
       e += (long long)gridDim.x * blockDim.x) {
    T v = 0;
    if (e < P.e_s) {                       // eta_y = y
      v = z[P.o_y + e];
    } else if (e < P.e_c) {                // eta_s = s^i - b'y^i
      const int i = (int)(e - P.e_s);
      const int c0 = P.ch_off[i], m = P.ch_off[i + 1] - c0;
      const T* y = z + P.o_y + P.yoff[i];
      T s = (i == 0) ? z[0] : z[P.o_s + i - 1];
      const int ly = (int)(P.yoff[i + 1] - P.yoff[i]);
      for (int k = 0; k < ly; ++k) s -= risk_b(P, i, c0, m, k) * y[k];
      v = s;
    } else if (e < P.e_q) {                // constraint rows of non-leaf nodes
      const long long f = e - P.e_c;
      const long long i = f / P.n_c;
      const int r = (int)(f % P.n_c);
      const int nball = P.has_ball ? nu : 0;
      if (r < P.nbx) v = P.gx[r] * z[P.o_x + i * nx + r];
      else if (r < P.nbx + P.nbu) v = P.gu[r - P.nbx] * z[P.o_u + i * nu + (r - P.nbx)];
      else if (r < P.nbox + nball) v = P.gu[r - P.nbox] * z[P.o_u + i * nu + (r - P.nbox)];
      else {                               // general row: [Gx Gu] (x^i, u^i)
        const T* G = P.Gg + (size_t)(r - P.nbox - nball) * (nx + nu);
        for (int k = 0; k < nx; ++k) v += G[k] * z[P.o_x + i * nx + k];
        for (int k = 0; k < nu; ++k) v += G[nx + k] * z[P.o_u + i * nu + k];
      }
    } else if (e < P.e_cN) {               // cost blocks of non-root nodes
      const long long f = e - P.e_q;
      const long long cm1 = f / P.W;
      const int k = (int)(f % P.W);
      const int a = P.anc[cm1 + 1];
      if (k < nx) {
        if (P.full) {
          const T* F = P.FQ + (size_t)cm1 * nx * nx + (size_t)k * nx;
          for (int q = 0; q < nx; ++q) v += F[q] * z[P.o_x + (long long)a * nx + q];
        } else {
          v = P.qh[cm1 * nx + k] * z[P.o_x + (long long)a * nx + k];
        }
      } else if (k < nx + nu) {
        if (P.full) {
          const T* F = P.FR + (size_t)cm1 * nu * nu + (size_t)(k - nx) * nu;
          for (int q = 0; q < nu; ++q) v += F[q] * z[P.o_u + (long long)a * nu + q];
        } else {
          v = P.rh[cm1 * nu + (k - nx)] * z[P.o_u + (long long)a * nu + (k - nx)];
        }
      } else {
        v = T(0.5) * z[P.o_tau + cm1];
        if (P.l1 != T(0)) v -= T(0.5) * P.l1 * z[P.o_th + a];   // (tau^c - lambda_0 theta^a)/2 (Prop. 2)
        if (P.soft) v -= T(0.5) * z[P.o_sg + a];                  // (tau^c - sigma^a)/2 (soft costs)
      }
    } else if (e < P.e_qN) {               // leaf constraint rows
      const long long f = e - P.e_cN;
      const long long j = f / P.n_cN;
      const int k = (int)(f % P.n_cN);
      const T* x = z + P.o_x + (P.n_nl + j) * nx;
      if (k < P.nbx) {
        v = P.gN[k] * x[k];
      } else {
        const T* G = P.GgN + (size_t)(k - P.nbx) * nx;
        for (int q = 0; q < nx; ++q) v += G[q] * x[q];
      }
    } else if (e >= P.e_sf) {              // soft-cost rows of non-leaf node i
      const int d = nx + nu;
      const long long f = e - P.e_sf;
      const long long i = f / (3 * d + 2);
      const int r = (int)(f % (3 * d + 2));
      const T* th = z + P.o_sth + i * d;
      if (r < d) v = P.smw[r] * th[r];                      // the cone: theta/s
      else if (r < d + 2) v = T(0.5) * z[P.o_sg + i];       // sigma/2, sigma/2
      else if (r < 2 * d + 2) v = th[r - d - 2];            // theta >= 0
      else {                                                 // theta - (x^i, u^i) >= slo
        const int k = r - 2 * d - 2;
        v = th[k] - ((k < nx) ? z[P.o_x + i * nx + k] : z[P.o_u + i * nu + (k - nx)]);
      }
    } else if (e >= P.e_l1) {              // l1 rows of non-leaf node i (Prop. 2)
      const int d = nx + nu;
      const long long f = e - P.e_l1;
      const long long i = f / (1 + 2 * d);
      const int r = (int)(f % (1 + 2 * d));
      const T* lam = z + P.o_lam + i * d;
      if (r == 0) {                        // theta - sum_k w_k lambda_k
        v = z[P.o_th + i];
        for (int k = 0; k < d; ++k) v -= P.l1w[k] * lam[k];
      } else {                             // lambda_k -/+ (x^i, u^i)_k
        const int k = (r - 1) % d;
        const T zk = (k < nx) ? z[P.o_x + i * nx + k] : z[P.o_u + i * nu + (k - nx)];
        v = (r <= d) ? lam[k] - zk : lam[k] + zk;
      }
    } else {                               // leaf cost blocks
      const long long f = e - P.e_qN;
      const long long j = f / (nx + 2);
      const int k = (int)(f % (nx + 2));
      const long long node = P.n_nl + j;
      if (k < nx) {
        if (P.full) {
          const T* F = P.FN + (size_t)j * nx * nx + (size_t)k * nx;
          for (int q = 0; q < nx; ++q) v += F[q] * z[P.o_x + node * nx + q];
        } else {
          v = P.qNh[j * nx + k] * z[P.o_x + node * nx + k];
        }
      } else {
        v = T(0.5) * z[P.o_s + node - 1];
      }
    }
    eta[e] = v;
  }
}

// z = L* eta (adjoint of Sec. 4.4, sums over siblings for x^i and u^i)
template <class T>
__global__ void k_apply_Lt(Prob<T> P, const int* __restrict__ ynode, const T* __restrict__ eta,
                           T* __restrict__ z) {
  const int nx = P.nx, nu = P.nu;
  const T* ey = eta + P.e_y;
  const T* es = eta + P.e_s;
  const T* ec = eta + P.e_c;
  const T* eq = eta + P.e_q;
  const T* ecN = eta + P.e_cN;
  const T* eqN = eta + P.e_qN;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < P.nz;
       e += (long long)gridDim.x * blockDim.x) {
    T v = 0;
    if (e == 0) {
      v = es[0];
    } else if (e < P.o_u) {                // x
      const long long f = e - P.o_x;
      const long long i = f / nx;
      const int k = (int)(f % nx);
      if (i < P.n_nl) {
        if (P.nbx) v = P.gx[k] * ec[i * P.n_c + k];
        for (int c = P.ch_off[i]; c < P.ch_off[i + 1]; ++c) {
          if (P.full) {
            const T* F = P.FQ + (size_t)(c - 1) * nx * nx + k;
            for (int q = 0; q < nx; ++q) v += F[(size_t)q * nx] * eq[(long long)(c - 1) * P.W + q];
          } else {
            v += P.qh[(long long)(c - 1) * nx + k] * eq[(long long)(c - 1) * P.W + k];
          }
        }
        const T* eg = ec + i * P.n_c + P.nbox + (P.has_ball ? nu : 0);
        for (int r = 0; r < P.n_g; ++r) v += P.GgT[(size_t)k * P.n_g + r] * eg[r];
        if (P.l1 != T(0)) {                 // l1 rows lambda - x, lambda + x
          const T* el = eta + P.e_l1 + i * (1 + 2 * (nx + nu));
          v += el[1 + (nx + nu) + k] - el[1 + k];
        }
        if (P.soft) v -= eta[P.e_sf + i * (3 * (nx + nu) + 2) + 2 * (nx + nu) + 2 + k];   // theta - x rows
      } else {
        const long long j = i - P.n_nl;
        if (P.nbx) v = P.gN[k] * ecN[j * P.n_cN + k];
        if (P.full) {
          const T* F = P.FN + (size_t)j * nx * nx + k;
          for (int q = 0; q < nx; ++q) v += F[(size_t)q * nx] * eqN[j * (nx + 2) + q];
        } else {
          v += P.qNh[j * nx + k] * eqN[j * (nx + 2) + k];
        }
        for (int r = 0; r < P.n_gN; ++r) v += P.GgNT[(size_t)k * P.n_gN + r] * ecN[j * P.n_cN + P.nbx + r];
      }
    } else if (e < P.o_y) {                // u
      const long long f = e - P.o_u;
      const long long i = f / nu;
      const int k = (int)(f % nu);
      if (P.nbu) v += P.gu[k] * ec[i * P.n_c + P.nbx + k];
      if (P.has_ball) v += P.gu[k] * ec[i * P.n_c + P.nbox + k];
      for (int c = P.ch_off[i]; c < P.ch_off[i + 1]; ++c) {
        if (P.full) {
          const T* F = P.FR + (size_t)(c - 1) * nu * nu + k;
          for (int q = 0; q < nu; ++q) v += F[(size_t)q * nu] * eq[(long long)(c - 1) * P.W + nx + q];
        } else {
          v += P.rh[(long long)(c - 1) * nu + k] * eq[(long long)(c - 1) * P.W + nx + k];
        }
      }
      const T* eg = ec + i * P.n_c + P.nbox + (P.has_ball ? nu : 0);
      for (int r = 0; r < P.n_g; ++r) v += P.GgT[(size_t)(nx + k) * P.n_g + r] * eg[r];
      if (P.l1 != T(0)) {                   // l1 rows lambda - u, lambda + u
        const T* el = eta + P.e_l1 + i * (1 + 2 * (nx + nu));
        v += el[1 + (nx + nu) + nx + k] - el[1 + nx + k];
      }
      if (P.soft) v -= eta[P.e_sf + i * (3 * (nx + nu) + 2) + 2 * (nx + nu) + 2 + nx + k];   // theta - u rows
    } else if (e < P.o_tau) {              // y
      const long long f = e - P.o_y;
      const int i = ynode[f];
      const int c0 = P.ch_off[i], m = P.ch_off[i + 1] - c0;
      const int k = (int)(f - P.yoff[i]);
      v = ey[f] - risk_b(P, i, c0, m, k) * es[i];
    } else if (e < P.o_s) {                // tau^c
      const long long cm1 = e - P.o_tau;
      v = T(0.5) * (eq[cm1 * P.W + nx + nu] + eq[cm1 * P.W + nx + nu + 1]);
    } else if (e < P.o_th) {               // s^c
      const long long cm1 = e - P.o_s;
      const long long c = cm1 + 1;
      if (c < P.n_nl) v = es[c];
      else {
        const long long j = c - P.n_nl;
        v = T(0.5) * (eqN[j * (nx + 2) + nx] + eqN[j * (nx + 2) + nx + 1]);
      }
    } else if (e < P.o_lam) {              // theta^i: its l1 row and the children's cost cones
      const long long i = e - P.o_th;
      v = eta[P.e_l1 + i * (1 + 2 * (nx + nu))];
      for (int c = P.ch_off[i]; c < P.ch_off[i + 1]; ++c)
        v -= T(0.5) * P.l1 * (eq[(long long)(c - 1) * P.W + nx + nu] + eq[(long long)(c - 1) * P.W + nx + nu + 1]);
    } else if (e >= P.o_sth) {             // theta^i_k of the soft costs: its cone entry and rows
      const int d = nx + nu;
      const long long f = e - P.o_sth;
      const long long i = f / d;
      const int k = (int)(f % d);
      const T* es_ = eta + P.e_sf + i * (3 * d + 2);
      v = P.smw[k] * es_[k] + es_[d + 2 + k] + es_[2 * d + 2 + k];
    } else if (e >= P.o_sg) {              // sigma^i: its cone and the children's cost cones
      const int d = nx + nu;
      const long long i = e - P.o_sg;
      const T* es_ = eta + P.e_sf + i * (3 * d + 2);
      v = T(0.5) * (es_[d] + es_[d + 1]);
      for (int c = P.ch_off[i]; c < P.ch_off[i + 1]; ++c)
        v -= T(0.5) * (eq[(long long)(c - 1) * P.W + nx + nu] + eq[(long long)(c - 1) * P.W + nx + nu + 1]);
    } else {                               // lambda^i_k: its l1 rows
      const int d = nx + nu;
      const long long f = e - P.o_lam;
      const long long i = f / d;
      const int k = (int)(f % d);
      const T* el = eta + P.e_l1 + i * (1 + 2 * d);
      v = -P.l1w[k] * el[0] + el[1 + k] + el[1 + d + k];
    }
    z[e] = v;
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 148 * 16) b = 148 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_scale_dyn(const SetupArgs& a, cudaStream_t s) {
  const long long tot = (long long)(a.n - 1) * (a.nx * a.nx + a.nx * a.nu + a.nx);
  k_scale_dyn<<<grid_for(tot, 256), 256, 0, s>>>(a.n, a.n_nl, a.nx, a.nu, a.anc, a.Sx, a.SxN,
                                                  a.Su, a.A, a.B, a.c, a.At, a.Bt, a.ct);
  return cudaGetLastError();
}

cudaError_t launch_alg1(const SetupArgs& a, const int* stage_off_host, int N, cudaStream_t s) {
  const long long tot = (long long)(a.n - a.n_nl) * a.nx * a.nx;
  k_leaf_P<<<grid_for(tot, 256), 256, 0, s>>>(a.n, a.n_nl, a.nx, a.P);
  for (int t = N - 1; t >= 0; --t) {
    const int p0 = stage_off_host[t], p1 = stage_off_host[t + 1];
    k_alg1_stage<<<p1 - p0, 256, 0, s>>>(p0, a.nx, a.nu, a.ch_off, a.At, a.Bt, a.P, a.K, a.Rt,
                                          a.Lc, a.Linv, a.Rinv, a.KA, a.BtP, a.PAb, a.Abar,
                                          a.err);
  }
  return cudaGetLastError();
}

cudaError_t launch_build(const SetupArgs& a, cudaStream_t s) {
  k_build_MB<<<grid_for((long long)(a.n - 1) * a.nx * a.ldB, 256), 256, 0, s>>>(
      a.n, a.nx, a.nu, a.ldB, a.anc, a.Abar, a.Bt, a.Rinv, a.MB);
  k_build_MF<<<grid_for((long long)(a.n - 1) * (a.nx + a.nu) * a.ldF, 256), 256, 0, s>>>(
      a.n, a.nx, a.nu, a.ldF, a.Abar, a.Bt, a.MF);
  k_build_MP_KT<<<grid_for((long long)a.n_nl * (a.nu * a.ldP + a.nx * a.ldK), 256), 256, 0, s>>>(
      a.n_nl, a.nx, a.nu, a.ldP, a.ldK, a.K, a.Rinv, a.MP, a.KT);
  k_build_Pc<<<grid_for((long long)(a.n - 1) * a.nx, 256), 256, 0, s>>>(a.n, a.nx, a.P, a.ct,
                                                                       a.Pc);
  k_build_kc<<<grid_for((long long)a.n_nl * (a.nx + a.nu), 256), 256, 0, s>>>(
      a.n_nl, a.nx, a.nu, a.ldB, a.ch_off, a.MB, a.Pc, a.kc);
  const long long tot = (long long)(a.n - 1) * (a.nx + a.nu) + (long long)(a.n - a.n_nl) * a.nx * 2 +
                        2 * a.nx + a.nu + (long long)a.n_nl * (a.nbx + a.nbu + 1);
  k_cost_con<<<grid_for(tot, 256), 256, 0, s>>>(
      a.n, a.n_nl, a.nx, a.nu, a.nbx, a.nbu, a.has_ball, a.anc, a.Sx, a.SxN, a.Su, a.a_con,
      a.a_conN, a.Qd, a.Rd, a.QNd, a.xlo, a.xhi, a.ulo, a.uhi, a.uball, a.qh, a.rh, a.qNh, a.gx,
      a.gu, a.gN, a.box_lo, a.box_hi, a.boxN_lo, a.boxN_hi, a.ball);
  return cudaGetLastError();
}

cudaError_t launch_norm_L(const SetupArgs& a, unsigned long long* out, cudaStream_t s) {
  k_norm_L<<<grid_for(a.n, 128), 128, 0, s>>>(a.n, a.n_nl, a.nx, a.nu, a.nbx,
                                                (a.nbu ? 1 : 0) + (a.has_ball ? 1 : 0), a.xu_shift, a.ys_block, a.soft_w, a.ch_off,
                                                a.prob, a.qh, a.rh, a.qNh, a.gx, a.gu, a.gN, out);
  return cudaGetLastError();
}

// dst[m][j * ldd + k] = src[m][k * lds + j] for k < rows, zero for rows <= k < ldd
template <class Dst>
__global__ void k_transpose(long long nmat, int rows, int cols, int lds, int ldd, const double* __restrict__ src,
                            Dst* __restrict__ dst) {
  const long long per = (long long)cols * ldd;
  const long long tot = nmat * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long m = e / per;
    const int j = (int)((e % per) / ldd), k = (int)(e % ldd);
    dst[e] = (k < rows) ? (Dst)src[m * rows * lds + (long long)k * lds + j] : (Dst)0;
  }
}

cudaError_t launch_transpose(const double* src, long long nmat, int rows, int cols, int lds, int ldd,
                             void* dst, int prec, cudaStream_t s) {
  const long long tot = nmat * cols * ldd;
  if (tot <= 0) return cudaSuccess;
  if (prec == 64)
    k_transpose<double><<<grid_for(tot, 256), 256, 0, s>>>(nmat, rows, cols, lds, ldd, src, (double*)dst);
  else
    k_transpose<float><<<grid_for(tot, 256), 256, 0, s>>>(nmat, rows, cols, lds, ldd, src, (float*)dst);
  return cudaGetLastError();
}

cudaError_t launch_convert_f64_f32(const double* a, float* b, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_convert<double, float><<<grid_for(n, 256), 256, 0, s>>>(n, a, b);
  return cudaGetLastError();
}
cudaError_t launch_convert_f32_f64(const float* a, double* b, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_convert<float, double><<<grid_for(n, 256), 256, 0, s>>>(n, a, b);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_apply_L(const Prob<T>& P, const int* ynode, const T* z, T* eta, cudaStream_t s) {
  k_apply_L<T><<<grid_for(P.neta, 256), 256, 0, s>>>(P, ynode, z, eta);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_apply_Lt(const Prob<T>& P, const int* ynode, const T* eta, T* z, cudaStream_t s) {
  k_apply_Lt<T><<<grid_for(P.nz, 256), 256, 0, s>>>(P, ynode, eta, z);
  return cudaGetLastError();
}
template cudaError_t launch_apply_L<float>(const Prob<float>&, const int*, const float*, float*, cudaStream_t);
template cudaError_t launch_apply_L<double>(const Prob<double>&, const int*, const double*, double*, cudaStream_t);
template cudaError_t launch_apply_Lt<float>(const Prob<float>&, const int*, const float*, float*, cudaStream_t);
template cudaError_t launch_apply_Lt<double>(const Prob<double>&, const int*, const double*, double*, cudaStream_t);

}  // namespace spock
