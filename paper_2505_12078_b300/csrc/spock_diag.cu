// spock_diag.cu -- the FP64 exit check of a solve (Sec. 5.3, "Termination").
//
// For an iterate v = (z, eta) and its image T(v) = (z+, eta+) under the
// Chambolle-Pock operator the paper measures epsilon-approximate optimality
// through
//   xi1 = (z - z+)/alpha - L*(eta - eta+),   xi2 = (eta - eta+)/alpha - L(z - z+)
// (Eq. xi1k and the line after it). Beside them this file computes the primal
// infeasibility ||L z+ - proj_S3(L z+)||_inf and the complementarity gap
// |<eta+, L z+> - sigma_S3(eta+)|, sigma the support function of S3 (Eq.
// S3-def): cone pieces contribute 0 (eta+ lies in the polar cone, which
// prox_{alpha g*} guarantees), boxes sum max(eta lo, eta hi), balls r ||eta||,
// translated second-order cones <eta, a> with a = (0, .., 1/2, -1/2).
//
// Everything runs in FP64 with fixed reduction orders (per-warp partials, then
// one block that combines them in index order), so a check is reproducible.
#include <cuda_runtime.h>
#include <math.h>

#include "spock_dev.cuh"
#include "spock_internal.h"

namespace spock {

namespace {

constexpr int kDiagBlocks = 148 * 4;   // grid of the block and element kernels
constexpr int kDiagThreads = 256;
constexpr int kDiagWarps = kDiagBlocks * kDiagThreads / 32;

// d = v - T(v)
__global__ void k_diff(long long nv, const double* __restrict__ v, const double* __restrict__ tv,
                       double* __restrict__ d) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nv; e += (long long)gridDim.x * blockDim.x)
    d[e] = v[e] - tv[e];
}

// per-block max of |d_z/alpha - Lt_de| (slot 0) and |d_eta/alpha - L_dz| (slot 1)
__global__ void k_xi(long long nz, long long neta, double alpha, const double* __restrict__ d,
                     const double* __restrict__ ltde, const double* __restrict__ ldz, double* __restrict__ part) {
  double m1 = 0.0, m2 = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nz + neta;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nz) m1 = fmax(m1, fabs(d[e] / alpha - ltde[e]));
    else m2 = fmax(m2, fabs(d[e] / alpha - ldz[e - nz]));
  }
  __shared__ double s1[32], s2[32];
  m1 = warp_max(m1);
  m2 = warp_max(m2);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { s1[w] = m1; s2[w] = m2; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    m1 = warp_max(lane < nw ? s1[lane] : 0.0);
    m2 = warp_max(lane < nw ? s2[lane] : 0.0);
    if (lane == 0) { part[2 * blockIdx.x] = m1; part[2 * blockIdx.x + 1] = m2; }
  }
}

// A translated second-order cone block of length dim at offset base of eta
// (a = (0.., 1/2, -1/2), last entry the scalar part): infeasibility of the
// block of L z+ and the block's terms of <eta+, L z+> and sigma(eta+).
__device__ __forceinline__ double cone_a(const double* acst, int e, int dim) {
  if (acst) return acst[e];
  return (e == dim - 2) ? 0.5 : ((e == dim - 1) ? -0.5 : 0.0);
}

__device__ void soc_diag(int lane, int dim, long long base, const double* __restrict__ lz,
                         const double* __restrict__ ep, const double* acst, double& inf, double& dot,
                         double& sig) {
  double n2 = 0.0, tt = 0.0;
  for (int e = lane; e < dim; e += 32) {
    const double a = cone_a(acst, e, dim);
    const double w = lz[base + e] - a;
    if (e < dim - 1) n2 += w * w;
    else tt = w;
  }
  const double nw = sqrt(warp_sum(n2));
  const double t = __shfl_sync(0xffffffffu, tt, (dim - 1) & 31);
  const int cs = (nw <= t) ? 0 : ((nw <= -t) ? 1 : 2);
  const double f = 0.5 * (nw + t);
  for (int e = lane; e < dim; e += 32) {
    const double a = cone_a(acst, e, dim);
    const double w = lz[base + e] - a;
    double p;
    if (cs == 0) p = w;
    else if (cs == 1) p = 0.0;
    else p = (e < dim - 1) ? w * (f / nw) : f;
    inf = fmax(inf, fabs(w - p));          // (lz - (a + p)) = w - p
    dot += ep[base + e] * lz[base + e];
    sig += ep[base + e] * a;
  }
}

// one warp per block of eta: non-leaf (y, s, constraint rows), non-root cost
// cone, leaf (constraint rows, cost cone). Partials per warp: max infeasibility,
// sum of eta+ * Lz+, sum of the support function terms.
__global__ void k_S3_diag(Prob<double> P, const double* __restrict__ lz, const double* __restrict__ ep,
                          double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nb = (long long)P.n_nl + (P.n - 1) + P.n_l;
  double inf = 0.0, dot = 0.0, sig = 0.0;
  for (long long b = gw; b < nb; b += nw) {
    if (b < P.n_nl) {
      const int i = (int)b;
      const int m = P.ch_off[i + 1] - P.ch_off[i];
      const long long ye = P.e_y + P.yoff[i];
      const int ly = (int)(P.yoff[i + 1] - P.yoff[i]), npos = risk_npos(P, m);
      for (int e = lane; e < ly; e += 32) {                 // (K^i)* = R^{npos}_+ x R
        const double x = lz[ye + e];
        const double p = (e < npos) ? fmax(x, 0.0) : x;
        inf = fmax(inf, fabs(x - p));
        dot += ep[ye + e] * x;
      }
      if (lane == 0) {                                      // R_+
        const long long is = P.e_s + i;
        const double x = lz[is];
        inf = fmax(inf, fabs(x - fmax(x, 0.0)));
        dot += ep[is] * x;
      }
      const long long ce = P.e_c + (long long)i * P.n_c;
      for (int e = lane; e < P.nbox; e += 32) {             // boxes
        const double x = lz[ce + e], h = ep[ce + e];
        const double lo = P.box_lo[(long long)i * P.nbox + e], hi = P.box_hi[(long long)i * P.nbox + e];
        inf = fmax(inf, fabs(x - fmin(fmax(x, lo), hi)));
        dot += h * x;
        sig += fmax(h * lo, h * hi);
      }
      if (P.has_ball) {                                     // ||u|| <= r rows
        double n2 = 0.0, h2 = 0.0;
        for (int k = lane; k < P.nu; k += 32) {
          const double x = lz[ce + P.nbox + k], h = ep[ce + P.nbox + k];
          n2 += x * x;
          h2 += h * h;
          dot += h * x;
        }
        const double nx_ = sqrt(warp_sum(n2)), nh = sqrt(warp_sum(h2));
        const double r = P.ball[i];
        if (lane == 0) sig += r * nh;
        // x - proj(x) = x (1 - r/||x||) outside the ball: its inf-norm is
        // max_k |x_k| (1 - r/||x||)
        if (nx_ > r) {
          double mx = 0.0;
          for (int k = lane; k < P.nu; k += 32) mx = fmax(mx, fabs(lz[ce + P.nbox + k]) * (1.0 - r / nx_));
          mx = warp_max(mx);
          if (lane == 0) inf = fmax(inf, mx);
        }
      }
      const long long ge = ce + P.nbox + (P.has_ball ? P.nu : 0);
      for (int e = lane; e < P.n_g; e += 32) {              // general rows: boxes
        const double x = lz[ge + e], h = ep[ge + e];
        const double lo = P.gen_lo[(long long)i * P.n_g + e], hi = P.gen_hi[(long long)i * P.n_g + e];
        inf = fmax(inf, fabs(x - fmin(fmax(x, lo), hi)));
        dot += h * x;
        sig += fmax(h * lo, h * hi);
      }
      if (P.soft) {                                         // soft-cost rows
        const int d = P.nx + P.nu;
        const long long se = P.e_sf + (long long)i * (3 * d + 2);
        soc_diag(lane, d + 2, se, lz, ep, nullptr, inf, dot, sig);   // translated cone (0, 1/2, -1/2)
        for (int e = lane; e < d; e += 32) {
          const double x0 = lz[se + d + 2 + e];             // theta >= 0: a cone, support 0
          inf = fmax(inf, fabs(x0 - fmax(x0, 0.0)));
          dot += ep[se + d + 2 + e] * x0;
          const double x1 = lz[se + 2 * d + 2 + e], h = ep[se + 2 * d + 2 + e];
          // [lo, inf): the support is h lo for h <= 0 and infinite above;
          // eta+ = min(0, eta_bar - alpha lo) is <= 0 exactly, but eta_bar -
          // alpha (eta_bar / alpha) can round to a few ulps above 0 where the
          // bound is inactive, so h is taken on the polar side, min(h, 0)
          const double lo = P.slo[e];
          inf = fmax(inf, fabs(x1 - fmax(x1, lo)));
          dot += h * x1;
          sig += fmin(h, 0.0) * lo;
        }
      }
      if (P.l1 != 0.0) {                                    // l1 rows (Prop. 2): R_+, support 0
        const int nr = 1 + 2 * (P.nx + P.nu);
        const long long le = P.e_l1 + (long long)i * nr;
        for (int e = lane; e < nr; e += 32) {
          const double x = lz[le + e];
          inf = fmax(inf, fabs(x - fmax(x, 0.0)));
          dot += ep[le + e] * x;
        }
      }
    } else if (b < P.n_nl + P.n - 1) {
      const long long c = b - P.n_nl + 1;
      soc_diag(lane, P.W, P.e_q + (c - 1) * P.W, lz, ep, P.acost ? P.acost + (c - 1) * P.W : nullptr, inf, dot,
               sig);
    } else {
      const long long jj = b - P.n_nl - (P.n - 1);
      const long long ce = P.e_cN + jj * P.n_cN;
      for (int e = lane; e < P.n_cN; e += 32) {
        const double x = lz[ce + e], h = ep[ce + e];
        const bool bx = e < P.nbx;
        const double lo = bx ? P.boxN_lo[jj * P.nx + e] : P.genN_lo[jj * P.n_gN + (e - P.nbx)];
        const double hi = bx ? P.boxN_hi[jj * P.nx + e] : P.genN_hi[jj * P.n_gN + (e - P.nbx)];
        inf = fmax(inf, fabs(x - fmin(fmax(x, lo), hi)));
        dot += h * x;
        sig += fmax(h * lo, h * hi);
      }
      soc_diag(lane, P.nx + 2, P.e_qN + jj * (P.nx + 2), lz, ep,
               P.acostN ? P.acostN + jj * (P.nx + 2) : nullptr, inf, dot, sig);
    }
  }
  inf = warp_max(inf);
  dot = warp_sum(dot);
  sig = warp_sum(sig);
  if (lane == 0) {
    part[3 * gw] = inf;
    part[3 * gw + 1] = dot;
    part[3 * gw + 2] = sig;
  }
}

// one block: combine the partials in index order. out = [xi1, xi2, infeas,
// gap, <eta+, L z+>, sigma_S3(eta+)]
__global__ void k_diag_final(int nwarps, const double* __restrict__ part, int nblk,
                             const double* __restrict__ part2, double* __restrict__ out) {
  __shared__ double s[4][kDiagThreads];
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
  for (int k = threadIdx.x; k < nwarps; k += blockDim.x) {
    a = fmax(a, part[3 * k]);
    b += part[3 * k + 1];
    c += part[3 * k + 2];
  }
  double m1 = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
    m1 = fmax(m1, part2[2 * k]);
    d = fmax(d, part2[2 * k + 1]);
  }
  s[0][threadIdx.x] = a; s[1][threadIdx.x] = b; s[2][threadIdx.x] = c; s[3][threadIdx.x] = m1;
  __shared__ double s4[kDiagThreads];
  s4[threadIdx.x] = d;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s[0][threadIdx.x] = fmax(s[0][threadIdx.x], s[0][threadIdx.x + h]);
      s[1][threadIdx.x] += s[1][threadIdx.x + h];
      s[2][threadIdx.x] += s[2][threadIdx.x + h];
      s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + h]);
      s4[threadIdx.x] = fmax(s4[threadIdx.x], s4[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s[3][0];
    out[1] = s4[0];
    out[2] = s[0][0];
    out[3] = fabs(s[1][0] - s[2][0]);
    out[4] = s[1][0];
    out[5] = s[2][0];
  }
}

}  // namespace

size_t diag_partials_doubles() { return (size_t)3 * kDiagWarps + (size_t)2 * kDiagBlocks + 8; }

// v, tv: FP64 (device) [n_v]. Scratch (device, FP64): d [n_v], ltde [n_z],
// ldz [n_eta], lz [n_eta], part [diag_partials_doubles()]. out6 (device) gets
// [xi1, xi2, infeas, gap, <eta+, L z+>, sigma_S3(eta+)].
cudaError_t launch_diagnostics(const Prob<double>& P, const int* ynode, const double* v, const double* tv,
                               double* d, double* ltde, double* ldz, double* lz, double* part, double* out6,
                               cudaStream_t s) {
  k_diff<<<kDiagBlocks, kDiagThreads, 0, s>>>(P.nv, v, tv, d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_apply_Lt<double>(P, ynode, d + P.nz, ltde, s)) != cudaSuccess) return e;
  if ((e = launch_apply_L<double>(P, ynode, d, ldz, s)) != cudaSuccess) return e;
  if ((e = launch_apply_L<double>(P, ynode, tv, lz, s)) != cudaSuccess) return e;
  double* part2 = part + 3 * kDiagWarps;
  k_xi<<<kDiagBlocks, kDiagThreads, 0, s>>>(P.nz, P.neta, (double)P.alpha, d, ltde, ldz, part2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_S3_diag<<<kDiagBlocks, kDiagThreads, 0, s>>>(P, lz, tv + P.nz, part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_diag_final<<<1, kDiagThreads, 0, s>>>(kDiagWarps, part, kDiagBlocks, part2, out6);
  return cudaGetLastError();
}

}  // namespace spock
