// spock_api.cu -- host runtime and C ABI of libspock (see include/spock.h).
//
// Owns the device memory of a problem: tree and schedule arrays, the FP64
// offline data, FP64 and FP32 copies of the per-iteration factors, and the
// solve buffers of each precision (allocated on first use). The offline part
// (Sec. 5.4 preconditioning, Alg. 1, ||L||) runs in FP64 kernels at creation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/spock.h"
#include "spock_dev.cuh"
#include "spock_internal.h"
#include "spock_cta.cuh"
#include "spock_problem.h"

using namespace spock;



namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? SPOCK_OK : SPOCK_EDEVICE; }

bool finite_arr(const double* a, long long n) {
  for (long long i = 0; i < n; ++i)
    if (!isfinite(a[i])) return false;
  return true;
}

// device copy of a host array in a setup-only allocation (nullptr for nullptr)
double* up_tmp(DevMem& tmp, const double* a, long long len) {
  if (!a) return nullptr;
  double* q = tmp.alloc<double>(len);
  if (q) cudaMemcpy(q, a, (size_t)len * sizeof(double), cudaMemcpyHostToDevice);
  return q;
}

// Largest eigenvalue of a symmetric m x m matrix (row-major) by cyclic Jacobi
// rotations (host, FP64; m <= 256, used once per problem).
double sym_max_eig(std::vector<double> a, int m) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        tot += a[(size_t)i * m + j] * a[(size_t)i * m + j];
        if (i != j) off += a[(size_t)i * m + j] * a[(size_t)i * m + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = a[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double app = a[(size_t)p * m + p], aqq = a[(size_t)q * m + q];
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < m; ++k) {   // columns p, q
          const double akp = a[(size_t)k * m + p], akq = a[(size_t)k * m + q];
          a[(size_t)k * m + p] = c * akp - sn * akq;
          a[(size_t)k * m + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {   // rows p, q
          const double apk = a[(size_t)p * m + k], aqk = a[(size_t)q * m + k];
          a[(size_t)p * m + k] = c * apk - sn * aqk;
          a[(size_t)q * m + k] = sn * apk + c * aqk;
        }
      }
  }
  double mx = 0.0;
  for (int i = 0; i < m; ++i) mx = std::max(mx, a[(size_t)i * m + i]);
  return mx;
}

// ||M||_2 of a rows x cols row-major matrix: sqrt of the largest eigenvalue of M'M
double mat_norm2(const std::vector<double>& M, int rows, int cols) {
  std::vector<double> g((size_t)cols * cols, 0.0);
  for (int i = 0; i < cols; ++i)
    for (int j = 0; j < cols; ++j) {
      double s = 0.0;
      for (int r = 0; r < rows; ++r) s += M[(size_t)r * cols + i] * M[(size_t)r * cols + j];
      g[(size_t)i * cols + j] = s;
    }
  return sqrt(std::max(0.0, sym_max_eig(g, cols)));
}

// Validate the tree (Sec. 3.2) and build the node arrays and sweep schedule.
int build_tree(spock_problem* p, int n, const int* anc, const double* prob, int tv) {
  if (n < 2 || !anc || !prob || anc[0] != -1) return SPOCK_EINVAL;
  std::vector<int> stage(n, 0);
  for (int i = 1; i < n; ++i) {
    if (anc[i] < 0 || anc[i] >= i) return SPOCK_EINVAL;
    if (anc[i] < anc[i - 1] && i > 1) return SPOCK_EINVAL;          // children contiguous
    stage[i] = stage[anc[i]] + 1;
    if (stage[i] < stage[i - 1]) return SPOCK_EINVAL;                // stage-major
    if (!(prob[i] > 0.0) || !(prob[i] <= 1.0 + 1e-12)) return SPOCK_EINVAL;
  }
  const int N = stage[n - 1];
  int n_nl = 0;
  while (n_nl < n && stage[n_nl] < N) ++n_nl;
  for (int i = n_nl; i < n; ++i)
    if (stage[i] != N) return SPOCK_EINVAL;
  std::vector<int> nch(n, 0);
  for (int i = 1; i < n; ++i) nch[anc[i]]++;
  for (int i = 0; i < n_nl; ++i)
    if (nch[i] == 0) return SPOCK_EINVAL;
  for (int i = n_nl; i < n; ++i)
    if (nch[i] != 0) return SPOCK_EINVAL;
  p->n = n; p->n_nl = n_nl; p->n_l = n - n_nl; p->N = N;
  p->anc.assign(anc, anc + n);
  p->ch_off.assign(n_nl + 1, 0);
  {
    int c = 1;
    for (int i = 0; i < n_nl; ++i) {
      p->ch_off[i] = c;
      c += nch[i];
    }
    p->ch_off[n_nl] = c;
    for (int i = 0; i < n_nl; ++i)
      for (int cc = p->ch_off[i]; cc < p->ch_off[i + 1]; ++cc)
        if (anc[cc] != i) return SPOCK_EINVAL;
  }
  for (int i = 0; i < n_nl; ++i) {
    double s = 0;
    for (int c = p->ch_off[i]; c < p->ch_off[i + 1]; ++c) s += prob[c];
    if (fabs(s - 1.0) > 1e-9) return SPOCK_EINVAL;
  }
  p->stage_off.assign(N + 2, 0);
  for (int t = 0, i = 0; t <= N; ++t) {
    p->stage_off[t] = i;
    while (i < n && stage[i] == t) ++i;
  }
  p->stage_off[N + 1] = n;
  p->yoff.assign(n_nl + 1, 0);
  for (int i = 0; i < n_nl; ++i) p->yoff[i + 1] = p->yoff[i] + (tv ? 3 * nch[i] + 2 : 2 * nch[i] + 1);
  p->n_y = p->yoff[n_nl];
  p->ynode.resize(p->n_y);
  for (int i = 0; i < n_nl; ++i)
    for (int k = p->yoff[i]; k < p->yoff[i + 1]; ++k) p->ynode[k] = i;
  // segments: chains of non-leaf nodes with a single non-leaf child
  auto is_top = [&](int i) { return i == 0 || nch[anc[i]] != 1; };
  auto is_bot = [&](int i) { return nch[i] != 1 || p->ch_off[i] >= n_nl; };
  std::vector<int> tops, bots, lens, seg_of(n_nl, -1);
  for (int i = 0; i < n_nl; ++i) {
    if (!is_top(i)) continue;
    int j = i, len = 1;
    seg_of[j] = (int)tops.size();
    while (!is_bot(j)) {
      j = p->ch_off[j];
      seg_of[j] = (int)tops.size();
      ++len;
    }
    tops.push_back(i); bots.push_back(j); lens.push_back(len);
  }
  const int ns = (int)tops.size();
  std::vector<int> level(ns, 0);
  for (int s = ns - 1; s >= 0; --s) {       // deeper tops come later in BFS order
    const int b = bots[s];
    int lv = 0;
    for (int c = p->ch_off[b]; c < p->ch_off[b + 1]; ++c)
      if (c < n_nl) lv = std::max(lv, level[seg_of[c]] + 1);
    level[s] = lv;
  }
  int L = 0;
  for (int s = 0; s < ns; ++s) L = std::max(L, level[s] + 1);
  p->lvl_off.assign(L + 1, 0);
  p->seg_top.clear(); p->seg_bot.clear(); p->seg_len.clear();
  int max_items = n;
  for (int l = 0; l < L; ++l) {
    p->lvl_off[l] = (int)p->seg_top.size();
    for (int s = 0; s < ns; ++s)
      if (level[s] == l) {
        p->seg_top.push_back(tops[s]); p->seg_bot.push_back(bots[s]); p->seg_len.push_back(lens[s]);
      }
  }
  p->lvl_off[L] = (int)p->seg_top.size();
  p->seg_off.clear(); p->seg_nodes.clear();
  for (size_t q = 0; q < p->seg_top.size(); ++q) {
    p->seg_off.push_back((int)p->seg_nodes.size());
    int j = p->seg_top[q];
    for (int k = 0; k < p->seg_len[q]; ++k) {
      p->seg_nodes.push_back(j);
      j = p->ch_off[j];
    }
  }
  p->seg_off.push_back((int)p->seg_nodes.size());
  p->max_items = max_items;
  return SPOCK_OK;
}

// largest eigenvalue of a symmetric 3 x 3 matrix by cyclic Jacobi rotations
// (each rotation zeroes one off-diagonal entry; the off-diagonal norm falls
// quadratically once small)
double sym3_max_eig(const double (&M)[3][3]) {
  double a[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) a[i][j] = M[i][j];
  for (int sweep = 0; sweep < 64; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-32 * dg) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < 3; ++k) {   // columns p, q
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - sn * akq;
          a[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {   // rows p, q
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - sn * aqk;
          a[q][k] = sn * apk + c * aqk;
        }
      }
  }
  return std::max(a[0][0], std::max(a[1][1], a[2][2]));
}

template <class T>
void fill_prob(spock_problem* p, Iter<T>& it, double alpha) {
  Prob<T>& P = it.P;
  P.n = p->n; P.n_nl = p->n_nl; P.n_l = p->n_l; P.N = p->N; P.nx = p->nx; P.nu = p->nu;
  P.n_c = p->n_c; P.n_cN = p->n_cN; P.nbx = p->nbx; P.nbu = p->nbu; P.nbox = p->nbox;
  P.has_ball = p->has_ball;
  P.nz = p->nz; P.neta = p->neta; P.nv = p->nv;
  P.o_x = p->o_x; P.o_u = p->o_u; P.o_y = p->o_y; P.o_tau = p->o_tau; P.o_s = p->o_s;
  P.e_y = p->e_y; P.e_s = p->e_s; P.e_c = p->e_c; P.e_q = p->e_q; P.e_cN = p->e_cN; P.e_qN = p->e_qN;
  P.W = p->nx + p->nu + 2;
  P.ldB = p->ldB; P.ldF = p->ldF; P.ldP = p->ldP; P.ldK = p->ldK;
  P.anc = p->d_anc; P.ch_off = p->d_ch_off; P.yoff = p->d_yoff;
  P.n_levels = (int)p->lvl_off.size() - 1;
  P.lvl_off = p->d_lvl_off; P.seg_top = p->d_seg_top; P.seg_bot = p->d_seg_bot; P.seg_len = p->d_seg_len;
  P.seg_off = p->d_seg_off; P.seg_nodes = p->d_seg_nodes; P.seg_info = p->d_seg_info;
  P.MB = it.MB; P.MF = it.MF; P.MP = it.MP; P.KT = it.KT; P.cvec = it.cvec; P.kc = it.kc;
  P.cta = it.cta; P.ldTB = it.ldTB; P.ldTF = it.ldTF; P.ldTK = it.ldTK; P.khB = it.khB; P.khF = it.khF;
  P.nbuf = it.nbuf; P.item_bytes = it.item_bytes; P.qslots = it.qslots; P.ldc = it.ldc;
  P.MBt = it.MBt; P.MFt = it.MFt; P.KTt = it.KTt;
  P.top_seg = p->d_top_seg; P.bot_seg = p->d_bot_seg;
  {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    P.seg_flag_off = nsm * 8;
  }
  P.qh = it.qh; P.rh = it.rh; P.qNh = it.qNh; P.gx = it.gx; P.gu = it.gu; P.gN = it.gN;
  P.box_lo = it.box_lo; P.box_hi = it.box_hi; P.boxN_lo = it.boxN_lo; P.boxN_hi = it.boxN_hi;
  P.ball = it.ball; P.prob = it.prob; P.avar = it.avar; P.x0s = it.x0s;
  P.full = p->full;
  P.FQ = it.FQ; P.FQT = it.FQT; P.FR = it.FR; P.FRT = it.FRT; P.FN = it.FN; P.FNT = it.FNT;
  P.acost = it.acost; P.acostN = it.acostN;
  P.n_g = p->n_g; P.n_gN = p->n_gN;
  P.Gg = it.Gg; P.GgT = it.GgT; P.GgN = it.GgN; P.GgNT = it.GgNT;
  P.gen_lo = it.gen_lo; P.gen_hi = it.gen_hi; P.genN_lo = it.genN_lo; P.genN_hi = it.genN_hi;
  P.alpha = (T)alpha;
  P.tv = p->tv; P.tvr = it.tvr;
  P.soft = p->soft; P.o_sg = p->o_sg; P.o_sth = p->o_sth; P.e_sf = p->e_sf; P.smw = it.smw; P.slo = it.slo;
  P.l1 = (T)p->l1; P.o_th = p->o_th; P.o_lam = p->o_lam; P.e_l1 = p->e_l1; P.l1w = it.l1w;
  P.qbuf = it.qbuf; P.dbuf = it.dbuf; P.hbuf = it.hbuf; P.ebuf = it.ebuf;
  P.mbb = it.mbb; P.mbf = it.mbf;
}

// Whole-CTA sweep layout (nx + nu <= 128): a column of a transposed factor is
// padded to a multiple of 16 bytes whose byte length is 32 or 96 mod 128, and
// the second thread of a column starts at a row whose byte offset is 16 mod 32;
// the four columns x two halves that one quarter-warp reads with 16-byte loads
// then fall on eight different 16-byte bank groups.
int cta_ld(int rows, int es) {
  const int q = 16 / es;
  int ld = (rows + q - 1) / q * q;
  while ((ld * es) % 128 != 32 && (ld * es) % 128 != 96) ld += q;
  return ld;
}
int cta_kh(int rows, int es) {
  int kh = (rows + 1) / 2;
  while ((kh * es) % 32 != 16) ++kh;
  return kh;
}

template <class T>
void cta_layout(spock_problem* p, Iter<T>& it) {
  const int nx = p->nx, nu = p->nu, es = (int)sizeof(T);
  it.cta = 0;
  if (!(p->tw == 8 && 2 * (nx + nu) <= kThreads)) return;
  it.ldTB = cta_ld(nx, es);
  it.ldTF = cta_ld(nx + nu, es);
  it.ldTK = cta_ld(nx, es);
  it.khB = cta_kh(nx, es);
  it.khF = cta_kh(nx + nu, es);
  const long long eb = (long long)(nx + nu) * it.ldTB;
  const long long ef = (long long)nu * it.ldTK + (long long)nx * it.ldTF;
  it.item_bytes = (int)((std::max(eb, ef) * es + 127) / 128 * 128);
  it.ldc = (nx + nu + 7) / 8 * 8;
  it.qslots = std::min(p->maxch, 8);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int prec = es == 8 ? 64 : 32;
  // static shared memory of the kernel and the per-warp / per-team views
  const long long fixed = 24 * 1024 + (long long)solver_smem_bytes(prec, p->tw, kThreads, nx + nu, 0) +
                          (long long)(2 + it.qslots) * it.ldc * es;
  const long long room = (long long)optin - fixed;
  const int nbuf = (int)std::min<long long>(4, room > 0 ? room / it.item_bytes : 0);
  if (nbuf < 2) return;
  it.nbuf = nbuf;
  it.cta = 1;
}

template <class T>
int alloc_iter(spock_problem* p, Iter<T>& it) {
  DevMem& m = p->mem;
  const int n = p->n, n_nl = p->n_nl, n_l = p->n_l, nx = p->nx, nu = p->nu;
  it.MB = m.alloc<T>((long long)(n - 1) * nx * p->ldB);
  it.MF = m.alloc<T>((long long)(n - 1) * (nx + nu) * p->ldF);
  it.MP = m.alloc<T>((long long)n_nl * nu * p->ldP);
  it.KT = m.alloc<T>((long long)n_nl * nx * p->ldK);
  it.cvec = m.alloc<T>((long long)(n - 1) * nx);
  it.kc = m.alloc<T>((long long)n_nl * (nx + nu));
  it.qh = m.alloc<T>((long long)(n - 1) * nx);
  it.rh = m.alloc<T>((long long)(n - 1) * nu);
  it.qNh = m.alloc<T>((long long)n_l * nx);
  it.gx = m.alloc<T>(nx); it.gu = m.alloc<T>(nu); it.gN = m.alloc<T>(nx);
  it.box_lo = m.alloc<T>((long long)n_nl * std::max(1, p->nbox));
  it.box_hi = m.alloc<T>((long long)n_nl * std::max(1, p->nbox));
  it.boxN_lo = m.alloc<T>((long long)n_l * nx);
  it.boxN_hi = m.alloc<T>((long long)n_l * nx);
  it.ball = m.alloc<T>(n_nl);
  it.prob = m.alloc<T>(n);
  it.avar = m.alloc<T>(n_nl);
  it.x0s = m.alloc<T>(nx);
  it.l1w = m.alloc<T>(nx + nu);
  it.tvr = m.alloc<T>(n_nl);
  if (p->soft) { it.smw = m.alloc<T>(nx + nu); it.slo = m.alloc<T>(nx + nu); }
  it.qbuf = m.alloc<T>((long long)n * nx);
  it.dbuf = m.alloc<T>((long long)n_nl * nu);
  it.hbuf = m.alloc<T>((long long)n_nl * nx);
  it.ebuf = m.alloc<T>((long long)n_nl * nu);
  if (p->full) {
    it.FQ = m.alloc<T>((long long)(n - 1) * nx * nx); it.FQT = m.alloc<T>((long long)(n - 1) * nx * nx);
    it.FR = m.alloc<T>((long long)(n - 1) * nu * nu); it.FRT = m.alloc<T>((long long)(n - 1) * nu * nu);
    it.FN = m.alloc<T>((long long)n_l * nx * nx); it.FNT = m.alloc<T>((long long)n_l * nx * nx);
  }
  if (p->has_lin) {
    it.acost = m.alloc<T>((long long)(n - 1) * (nx + nu + 2));
    it.acostN = m.alloc<T>((long long)n_l * (nx + 2));
  }
  if (p->n_g) {
    it.Gg = m.alloc<T>((long long)p->n_g * (nx + nu)); it.GgT = m.alloc<T>((long long)p->n_g * (nx + nu));
    it.gen_lo = m.alloc<T>((long long)n_nl * p->n_g); it.gen_hi = m.alloc<T>((long long)n_nl * p->n_g);
  }
  if (p->n_gN) {
    it.GgN = m.alloc<T>((long long)p->n_gN * nx); it.GgNT = m.alloc<T>((long long)p->n_gN * nx);
    it.genN_lo = m.alloc<T>((long long)n_l * p->n_gN); it.genN_hi = m.alloc<T>((long long)n_l * p->n_gN);
  }
  cta_layout<T>(p, it);
  if (it.cta) {
    it.MBt = m.alloc<T>((long long)(n - 1) * (nx + nu) * it.ldTB);
    it.MFt = m.alloc<T>((long long)(n - 1) * nx * it.ldTF);
    it.KTt = m.alloc<T>((long long)n_nl * nu * it.ldTK);
    it.mb_bytes = mailbox_bytes(n, nx + nu, sizeof(T));
    it.mbb = m.alloc<unsigned long long>((long long)(it.mb_bytes / 8));
    it.mbf = m.alloc<unsigned long long>((long long)(it.mb_bytes / 8));
  }
  return m.failed ? SPOCK_ENOMEM : SPOCK_OK;
}


__global__ void k_scale_x0(int nx, const double* __restrict__ x0, const double* __restrict__ Sx,
                           double* __restrict__ o64, float* __restrict__ o32) {
  for (int k = threadIdx.x; k < nx; k += blockDim.x) {
    const double v = Sx[k] * x0[k];
    o64[k] = v;
    o32[k] = (float)v;
  }
}

// x = x~ / S, u = u~ / Su from the z part of T(v)
template <class T>
__global__ void k_unscale(int n, int n_nl, int nx, int nu, long long o_x, long long o_u,
                          const T* __restrict__ z, const double* __restrict__ Sx,
                          const double* __restrict__ SxN, const double* __restrict__ Su,
                          double* __restrict__ xo, double* __restrict__ uo, double* __restrict__ risk) {
  const long long nX = (long long)n * nx, nU = (long long)n_nl * nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nX + nU + 1;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nX) {
      const long long i = e / nx;
      const int k = (int)(e % nx);
      if (xo) xo[e] = (double)z[o_x + e] / ((i >= n_nl) ? SxN[k] : Sx[k]);
    } else if (e < nX + nU) {
      const long long f = e - nX;
      if (uo) uo[f] = (double)z[o_u + f] / Su[f % nu];
    } else {
      *risk = (double)z[0];
    }
  }
}

// warps per team of the sweeps; the column-split mat-vecs need
// 2 * 32 * tw >= nx + nu (at most two output columns per thread)
int pick_tw(int nx, int nu) {
  const int d = nx + nu;
  if (2 * d <= 256 && d >= 32) return 8;   // whole-CTA sweeps (two threads per column)
  if (d >= 96) return 8;
  if (d >= 48) return 4;
  if (d >= 24) return 2;
  return 1;
}

// Bytes of the largest per-node matrix streamed through shared memory by the
// sweeps, or 0 when two of them per team do not fit (then the sweeps read the
// matrices from global memory).
template <class T>
int pipe_bytes_for(const spock_problem* p) {
  if ((sizeof(T) == 8 ? p->f64.cta : p->f32.cta)) return 0;   // the whole-CTA sweeps have their ring
  // backward item: MB; forward item: [KT | MF]
  const long long e = std::max((long long)p->nx * p->ldB,
                               (long long)(p->nx + p->nu) * p->ldF + (long long)p->nx * p->ldK);
  const int b = (int)(e * (long long)sizeof(T));
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int prec = sizeof(T) == 8 ? 64 : 32;
  const size_t need = solver_smem_bytes(prec, p->tw, kThreads, p->nx + p->nu, b) + 4096;
  return (need <= (size_t)optin) ? b : 0;
}

// cycle probes of the last solve (see SolveCtl::prof)
static unsigned long long g_last_prof[16];
// bounds-checked build: the site of the last failed index check (0: none)
static int g_last_check = 0;

// test hook of spock_debug_wait_fault: extra CTAs the grid barriers of a
// single-problem launch wait for, and the limit of one barrier wait
static int g_phantom = 0;
static unsigned long long g_wait_ns = 0;

template <class T>
int run_solver(spock_problem* p, Iter<T>& it, const SolveOpts& so_in, cudaStream_t st, SolveCtl* h_ctl,
               float* ms) {
  int rc = ensure_bufs(p, it);
  if (rc) return rc;
  SolveOpts so = so_in;
  so.phantom = g_phantom;
  so.wait_ns = g_wait_ns;
  const int prec = sizeof(T) == 8 ? 64 : 32;
  it.P.pipe_bytes = p->use_pipe ? pipe_bytes_for<T>(p) : 0;
  int maxg = 0;
  if (solver_max_grid(prec, p->tw, kThreads, p->nx + p->nu, it.P.pipe_bytes, cta_smem_bytes(it.P), &maxg) ||
      maxg <= 0)
    return SPOCK_EDEVICE;
  const int teams = (kThreads / 32) / p->tw;
  int grid = (p->max_items + teams - 1) / teams;
  if (grid > maxg) grid = maxg;
  if (grid < 1) grid = 1;
  if (cudaMemsetAsync(it.sb.ctl, 0, sizeof(SolveCtl), st) != cudaSuccess) return SPOCK_EDEVICE;
  if (cudaMemsetAsync(it.sb.flags, 0, sizeof(unsigned) * (it.P.seg_flag_off + p->seg_top.size()), st) !=
      cudaSuccess)
    return SPOCK_EDEVICE;
  if (it.mbb && (cudaMemsetAsync(it.mbb, 0, it.mb_bytes, st) != cudaSuccess ||
                 cudaMemsetAsync(it.mbf, 0, it.mb_bytes, st) != cudaSuccess))
    return SPOCK_EDEVICE;
  cudaEventRecord(p->ev0, st);
  cudaError_t e = launch_solve<T>(it.P, it.sb, so, p->tw, grid, kThreads, st);
  if (e != cudaSuccess) return SPOCK_EDEVICE;
  cudaEventRecord(p->ev1, st);
  if (cudaMemcpyAsync(h_ctl, it.sb.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SPOCK_EDEVICE;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPOCK_EDEVICE;
  if (ms) cudaEventElapsedTime(ms, p->ev0, p->ev1);
  for (int q = 0; q < 16; ++q) g_last_prof[q] = h_ctl->prof[q];
  if (h_ctl->check_site) {   // bounds-checked build: an index check failed
    g_last_check = h_ctl->check_site;
    if (getenv("SPOCK_DEBUG")) fprintf(stderr, "spock: index check %d failed\n", h_ctl->check_site);
    return SPOCK_EDEVICE;
  }
  if (h_ctl->status < 0) {
    if (getenv("SPOCK_DEBUG"))
      fprintf(stderr, "spock: device wait gave up: cta %d barrier 0x%x parity %d site %d\n",
              h_ctl->diag[0], h_ctl->diag[1], h_ctl->diag[2], h_ctl->diag[3]);
    return SPOCK_ETIMEOUT;
  }
  return SPOCK_OK;
}

template <class T>
T* buf_index(SolveBufs<T>& b, int i) {
  return i == 0 ? b.V : i == 1 ? b.TV : i == 2 ? b.VT : b.TVT;
}

}  // namespace

// One evaluation of T whose scratch (control block, barrier flags, reduction
// partials and the sweep vectors q, d, h, e) is carved from a caller-provided
// device region instead of the problem's own buffers. Allocates nothing.
// Returns SPOCK_EUNSUPPORTED when the region is too small.
namespace spock {
int op_T_with_scratch(spock_problem* p, int precision, const void* v_in, void* v_out,
                      double* stats, cudaStream_t st, unsigned char* scratch, size_t bytes) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPOCK_EDEVICE;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t maxg = (size_t)nsm * 8;
  const size_t w = (precision == 64) ? 8 : 4;
  size_t off = 0;
  const size_t o_ctl = off;   off += al(sizeof(SolveCtl));
  const size_t nflags = maxg + p->seg_top.size();   // barrier flags, then segment flags
  const size_t o_flags = off; off += al(nflags * sizeof(unsigned));
  const size_t o_part = off;  off += al(2 * maxg * NRED * sizeof(double));
  const size_t o_q = off;     off += al((size_t)p->n * p->nx * w);
  const size_t o_d = off;     off += al((size_t)p->n_nl * p->nu * w);
  const size_t o_h = off;     off += al((size_t)p->n_nl * p->nx * w);
  const size_t o_e = off;     off += al((size_t)p->n_nl * p->nu * w);
  const size_t mbx = mailbox_bytes(p->n, p->nx + p->nu, w);
  const size_t o_mb = off;    off += al(2 * mbx);   // sweep mailboxes (zeroed below)
  if (off > bytes) return SPOCK_EUNSUPPORTED;
  SolveCtl* ctl = reinterpret_cast<SolveCtl*>(scratch + o_ctl);
  unsigned* flags = reinterpret_cast<unsigned*>(scratch + o_flags);
  // what must start at zero: the control block (barrier state, error word) and the flags
  if (cudaMemsetAsync(ctl, 0, sizeof(SolveCtl), st) != cudaSuccess) return SPOCK_EDEVICE;
  if (cudaMemsetAsync(flags, 0, nflags * sizeof(unsigned), st) != cudaSuccess) return SPOCK_EDEVICE;
  if (cudaMemsetAsync(scratch + o_mb, 0, 2 * mbx, st) != cudaSuccess) return SPOCK_EDEVICE;
  SolveOpts so{1e300, 0, 1, 2, 1e-10};
  const int teams = (kThreads / 32) / p->tw;
  cudaError_t e;
  int maxgrid = 0;
  if (precision == 64) {
    Prob<double> P = p->f64.P;
    P.qbuf = reinterpret_cast<double*>(scratch + o_q);
    P.dbuf = reinterpret_cast<double*>(scratch + o_d);
    P.hbuf = reinterpret_cast<double*>(scratch + o_h);
    P.ebuf = reinterpret_cast<double*>(scratch + o_e);
    P.mbb = reinterpret_cast<unsigned long long*>(scratch + o_mb);
    P.mbf = reinterpret_cast<unsigned long long*>(scratch + o_mb + mbx);
    P.pipe_bytes = p->use_pipe ? pipe_bytes_for<double>(p) : 0;
    if (solver_max_grid(64, p->tw, kThreads, p->nx + p->nu, P.pipe_bytes, cta_smem_bytes(P), &maxgrid) ||
        maxgrid <= 0)
      return SPOCK_EDEVICE;
    int grid = std::min((p->max_items + teams - 1) / teams, std::min(maxgrid, (int)maxg));
    SolveBufs<double> B{};
    B.V = (double*)v_in; B.TV = (double*)v_out;
    B.partials = reinterpret_cast<double*>(scratch + o_part);
    B.flags = flags; B.ctl = ctl;
    e = launch_solve<double>(P, B, so, p->tw, std::max(grid, 1), kThreads, st);
  } else {
    Prob<float> P = p->f32.P;
    P.qbuf = reinterpret_cast<float*>(scratch + o_q);
    P.dbuf = reinterpret_cast<float*>(scratch + o_d);
    P.hbuf = reinterpret_cast<float*>(scratch + o_h);
    P.ebuf = reinterpret_cast<float*>(scratch + o_e);
    P.mbb = reinterpret_cast<unsigned long long*>(scratch + o_mb);
    P.mbf = reinterpret_cast<unsigned long long*>(scratch + o_mb + mbx);
    P.pipe_bytes = p->use_pipe ? pipe_bytes_for<float>(p) : 0;
    if (solver_max_grid(32, p->tw, kThreads, p->nx + p->nu, P.pipe_bytes, cta_smem_bytes(P), &maxgrid) ||
        maxgrid <= 0)
      return SPOCK_EDEVICE;
    int grid = std::min((p->max_items + teams - 1) / teams, std::min(maxgrid, (int)maxg));
    SolveBufs<float> B{};
    B.V = (float*)v_in; B.TV = (float*)v_out;
    B.partials = reinterpret_cast<double*>(scratch + o_part);
    B.flags = flags; B.ctl = ctl;
    e = launch_solve<float>(P, B, so, p->tw, std::max(grid, 1), kThreads, st);
  }
  if (e != cudaSuccess) return SPOCK_EDEVICE;
  SolveCtl h{};
  if (cudaMemcpyAsync(&h, ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SPOCK_EDEVICE;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPOCK_EDEVICE;
  if (h.check_site) { g_last_check = h.check_site; return SPOCK_EDEVICE; }
  if (h.status < 0) return SPOCK_ETIMEOUT;
  if (stats)
    for (int k = 0; k < 8; ++k) stats[k] = h.stats[k];
  return SPOCK_OK;
}
}  // namespace spock

namespace spock {
static int sm_count() {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}
static inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

long long solve_buffer_bytes(const spock_problem* p, int precision) {
  const size_t w = precision == 64 ? 8 : 4;
  const size_t nv = (size_t)p->nv, nvp = (size_t)((p->nv + 3) & ~3LL);
  const size_t nsm = (size_t)sm_count();
  return (long long)(7 * al256(nv * w) + 2 * al256(3 * nvp * w) + al256(2 * nsm * 8 * NRED * sizeof(double)) +
                     al256((nsm * 8 + p->seg_top.size()) * sizeof(unsigned)) + al256(sizeof(SolveCtl)));
}

template <class T>
int ensure_bufs(spock_problem* p, Iter<T>& it) {
  if (it.have_bufs) return SPOCK_OK;
  const long long nv = p->nv;
  const size_t w = sizeof(T);
  const size_t nsm = (size_t)sm_count();
  const size_t bytes = (size_t)solve_buffer_bytes(p, w == 8 ? 64 : 32);
  void* blk = nullptr;
  if (cudaMalloc(&blk, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SPOCK_ENOMEM;
  }
  unsigned char* q = static_cast<unsigned char*>(blk);
  auto take = [&](size_t n) {
    unsigned char* r = q;
    q += al256(n);
    return r;
  };
  SolveBufs<T>& b = it.sb;
  const long long nvp = (nv + 3) & ~3LL;   // 16-byte aligned slots
  b.V = (T*)take(nv * w); b.TV = (T*)take(nv * w); b.VT = (T*)take(nv * w); b.TVT = (T*)take(nv * w);
  b.PSI = (T*)take(nv * w); b.VP = (T*)take(nv * w); b.RP = (T*)take(nv * w);
  b.sstride = nvp;
  b.S = (T*)take(3 * nvp * w); b.Y = (T*)take(3 * nvp * w);
  b.partials = (double*)take(2 * nsm * 8 * NRED * sizeof(double));
  b.flags = (unsigned*)take((nsm * 8 + p->seg_top.size()) * sizeof(unsigned));   // + segment flags
  b.ctl = (SolveCtl*)take(sizeof(SolveCtl));
  it.sb_block = blk;
  cudaMemset(b.V, 0, nv * w);
  cudaMemset(b.S, 0, 3 * nvp * w);
  cudaMemset(b.Y, 0, 3 * nvp * w);
  it.have_bufs = true;
  return cuda_err(cudaGetLastError());
}

template <class T>
void release_bufs(Iter<T>& it) {
  if (it.sb_block) cudaFree(it.sb_block);
  it.sb_block = nullptr;
  it.sb = SolveBufs<T>{};
  it.have_bufs = false;
}
template void release_bufs<float>(Iter<float>&);
template void release_bufs<double>(Iter<double>&);
template int ensure_bufs<float>(spock_problem*, Iter<float>&);
template int ensure_bufs<double>(spock_problem*, Iter<double>&);
}  // namespace spock

namespace {
// xi1, xi2, infeasibility, gap, <eta+, L z+>, sigma_S3(eta+) of an FP64 pair
// (v, T(v)) into out6 (host); scratch: the FP64 solve buffers VP, RP, S
int diag_run(spock_problem* p, const double* v, const double* tv, cudaStream_t st, double* out6) {
  int rc = ensure_bufs(p, p->f64);
  if (rc) return rc;
  const size_t np = diag_partials_doubles();
  if (!p->d_diag_part) {
    p->d_diag_part = p->mem.alloc<double>((long long)np + 8);
    if (!p->d_diag_part) return SPOCK_ENOMEM;
  }
  SolveBufs<double>& b = p->f64.sb;
  double* dout = p->d_diag_part + np;
  if (launch_diagnostics(p->f64.P, p->d_ynode, v, tv, b.VP, b.RP, b.S, b.S + b.sstride, p->d_diag_part, dout,
                         st) != cudaSuccess)
    return SPOCK_EDEVICE;
  if (cudaMemcpyAsync(out6, dout, 6 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SPOCK_EDEVICE;
  return cuda_err(cudaStreamSynchronize(st));
}
}  // namespace

namespace spock {
int check_fp64(spock_problem* p, int precision, const void* v, cudaStream_t st, double* out7) {
  int rc = ensure_bufs(p, p->f64);
  if (rc) return rc;
  const long long nv = p->nv;
  cudaError_t e;
  if (precision == 32) e = launch_convert_f32_f64((const float*)v, p->f64.sb.VT, nv, st);
  else if (v != p->f64.sb.VT) e = cudaMemcpyAsync(p->f64.sb.VT, v, nv * 8, cudaMemcpyDeviceToDevice, st);
  else e = cudaSuccess;
  if (e != cudaSuccess) return SPOCK_EDEVICE;
  Iter<double> it = p->f64;
  it.sb.V = p->f64.sb.VT;
  it.sb.TV = p->f64.sb.TVT;
  SolveOpts s1{1e300, 0, 1, 2, 1e-10};
  SolveCtl h2{};
  rc = run_solver<double>(p, it, s1, st, &h2, nullptr);
  if (rc) return rc;
  out7[0] = h2.res_inf;
  return diag_run(p, p->f64.sb.VT, p->f64.sb.TVT, st, out7 + 1);
}
}  // namespace spock

namespace spock {
// buffers of the centred FP32 iteration (first use, one allocation)
static int ensure_ctr(spock_problem* p) {
  if (p->ctr_block) return SPOCK_OK;
  const size_t ne = (size_t)p->neta, nz = (size_t)p->nz;
  size_t nzero = (size_t)(p->n - 1) * p->nx;
  nzero = std::max(nzero, (size_t)p->n_nl * (p->nx + p->nu));
  nzero = std::max(nzero, (size_t)p->nx);
  const size_t bytes = 2 * al256(ne * 8) + al256(nz * 4) + al256(nzero * 4);
  void* blk = nullptr;
  if (cudaMalloc(&blk, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SPOCK_ENOMEM;
  }
  unsigned char* q = static_cast<unsigned char*>(blk);
  p->d_ctrA = (double*)q; q += al256(ne * 8);
  p->d_ctrB = (double*)q; q += al256(ne * 8);
  p->d_cz = (float*)q;    q += al256(nz * 4);
  p->d_zero32 = (float*)q;
  if (cudaMemset(p->d_zero32, 0, nzero * 4) != cudaSuccess) {
    cudaFree(blk);
    return SPOCK_EDEVICE;
  }
  p->ctr_block = blk;
  p->ctr_bytes = (long long)bytes;
  return SPOCK_OK;
}

// Data of the centre c (FP64, n_v): T(c) into the FP64 solve buffer TV, L z_c
// into VT, then cz, A, B; res_c = ||c - T(c)||_inf in FP64. Needs the FP64
// solve buffers and the centre buffers.
static int centre_at(spock_problem* p, const double* c, cudaStream_t st, double* res_c) {
  double* tc = p->f64.sb.TV;
  double* lz = p->f64.sb.VT;
  Iter<double> e64 = p->f64;
  e64.sb.V = const_cast<double*>(c);
  e64.sb.TV = tc;
  const SolveOpts s1{1e300, 0, 1, 2, 1e-10};   // one evaluation of T
  SolveCtl h1{};
  int rc = run_solver<double>(p, e64, s1, st, &h1, nullptr);
  if (rc) return rc;
  *res_c = h1.res_inf;
  if (launch_apply_L<double>(p->f64.P, p->d_ynode, c, lz, st) != cudaSuccess) return SPOCK_EDEVICE;
  if (launch_centre(p->f64.P, c, tc, lz, p->alpha, p->d_cz, p->d_ctrA, p->d_ctrB, st) != cudaSuccess)
    return SPOCK_EDEVICE;
  return SPOCK_OK;
}

// the FP32 descriptor of the centred form: the linear part of prox_f (zeros
// for x0, c and the constant of the backward recursion) and the centre's data
static Iter<float> centred_iter(spock_problem* p) {
  Iter<float> it = p->f32;
  it.P.lin = 1;
  it.P.cvec = p->d_zero32;
  it.P.kc = p->d_zero32;
  it.P.x0s = p->d_zero32;
  it.P.cz = p->d_cz;
  it.P.ctrA = p->d_ctrA;
  it.P.ctrB = p->d_ctrB;
  it.P.ctr_al = p->alpha;
  it.P.ctr_ial = 1.0 / p->alpha;
  return it;
}

// one FP32 evaluation of the centred map: out = T(c + delta) - c
int op_T_centred(spock_problem* p, const double* c, const float* delta, float* out, double* stats,
                 cudaStream_t st) {
  int rc = ensure_bufs(p, p->f64);
  if (rc) return rc;
  rc = ensure_bufs(p, p->f32);
  if (rc) return rc;
  rc = ensure_ctr(p);
  if (rc) return rc;
  double res_c = 0.0;
  rc = centre_at(p, c, st, &res_c);
  if (rc) return rc;
  Iter<float> it = centred_iter(p);
  it.sb.V = const_cast<float*>(delta);
  it.sb.TV = out;
  const SolveOpts s1{1e300, 0, 1, 2, 1e-10};
  SolveCtl h{};
  rc = run_solver<float>(p, it, s1, st, &h, nullptr);
  if (rc) return rc;
  if (stats)
    for (int k = 0; k < 8; ++k) stats[k] = h.stats[k];
  return SPOCK_OK;
}

// The centred FP32 iteration (spock_solve_opts.recentre > 0): segments of the
// FP32 SPOCK iteration on delta = v - c, each started from delta = 0 at a new
// FP64 centre c and stopped once its FP32 residual is below recentre times the
// centre's FP64 residual (or tol); the FP64 residual of the centre, from one
// FP64 evaluation of T, is the stopping test. Outputs and the exit check come
// from the final centre and its FP64 image.
static int solve_centred(spock_problem* p, const spock_solve_opts& o, const SolveOpts& so, cudaStream_t st,
                         double* x_out, double* u_out, SolveCtl& tot, double& res_c, double (&diag6)[6],
                         int& n_ctr, double& kern_ms) {
  int rc = ensure_bufs(p, p->f64);
  if (rc) return rc;
  rc = ensure_bufs(p, p->f32);
  if (rc) return rc;
  rc = ensure_ctr(p);
  if (rc) return rc;
  const long long nv = p->nv;
  double* c = p->f64.sb.V;     // the centre (the FP64 iterate)
  double* tc = p->f64.sb.TV;   // T(c)
  if (!o.warm_start && cudaMemsetAsync(c, 0, nv * 8, st) != cudaSuccess) return SPOCK_EDEVICE;
  Iter<float> it = centred_iter(p);
  int left = o.max_iters;
  n_ctr = 0;
  kern_ms = 0.0;
  tot = SolveCtl{};
  tot.status = 1;
  for (;;) {
    rc = centre_at(p, c, st, &res_c);
    if (rc) return rc;
    ++n_ctr;
    ++tot.n_T;
    if (res_c <= o.tol) {
      tot.status = 0;
      break;
    }
    if (left <= 0) break;
    if (cudaMemsetAsync(it.sb.V, 0, nv * 4, st) != cudaSuccess) return SPOCK_EDEVICE;
    SolveOpts sg = so;
    sg.tol = std::max(o.tol, o.recentre * res_c);
    sg.max_iters = left;
    SolveCtl h{};
    float seg_ms = 0.f;
    rc = run_solver<float>(p, it, sg, st, &h, &seg_ms);
    if (rc) return rc;
    kern_ms += seg_ms;
    tot.iters += h.iters; tot.n_T += h.n_T; tot.n_K0 += h.n_K0; tot.n_K1 += h.n_K1; tot.n_K2 += h.n_K2;
    tot.n_fb += h.n_fb; tot.n_bt += h.n_bt;
    for (int q = 0; q < 16; ++q) tot.prof[q] += h.prof[q];
    left -= h.iters;
    if (launch_centre_move(nv, c, buf_index(it.sb, h.final_v), st) != cudaSuccess) return SPOCK_EDEVICE;
  }
  tot.res_inf = res_c;
  k_unscale<double><<<64, 256, 0, st>>>(p->n, p->n_nl, p->nx, p->nu, p->o_x, p->o_u, tc, p->d_Sx, p->d_SxN,
                                       p->d_Su, x_out, u_out, p->d_out_risk);
  if (launch_centre_to_f32(nv, c, p->f32.sb.V, st) != cudaSuccess) return SPOCK_EDEVICE;
  return diag_run(p, c, tc, st, diag6);
}
}  // namespace spock

extern "C" {

int spock_version(void) { return 3; }

int spock_debug_last_check(void) {
#ifdef SPOCK_CHECKED
  return g_last_check;
#else
  return -1;
#endif
}

int spock_debug_wait_fault(int phantom_ctas, double wait_limit_s) {
  if (phantom_ctas < 0 || phantom_ctas > 4 || !(wait_limit_s >= 0.0) || wait_limit_s > 10.0) return SPOCK_EINVAL;
  g_phantom = phantom_ctas;
  g_wait_ns = (unsigned long long)(wait_limit_s * 1e9);
  return SPOCK_OK;
}

const char* spock_status_str(int s) {
  switch (s) {
    case SPOCK_OK: return "ok";
    case SPOCK_MAXITER: return "not converged within max_iters";
    case SPOCK_PARTIAL: return "only some plants admitted (device memory)";
    case SPOCK_EINVAL: return "invalid argument";
    case SPOCK_ENOMEM: return "out of device memory";
    case SPOCK_ENOTPD: return "R~ = I + sum B'PB not positive definite";
    case SPOCK_EDEVICE: return "CUDA runtime error";
    case SPOCK_ETIMEOUT: return "device-side wait ran out of time";
    case SPOCK_EUNSUPPORTED: return "sizes beyond the compiled limits";
    default: return "unknown status";
  }
}

void spock_solve_opts_default(spock_solve_opts* o) {
  if (!o) return;
  o->precision = 64;
  o->tol = 1e-4;
  o->max_iters = 5000;
  o->max_backtracks = 30;
  o->method = 0;
  o->warm_start = 0;
  o->fp64_check = 1;
  o->aa_mode = 0;
  o->recentre = 0.1;
}

int spock_problem_create(const spock_problem_desc* d, spock_problem** out) {
  if (!out) return SPOCK_EINVAL;
  *out = nullptr;
  if (!d || !d->A || !d->B || !d->Q || !d->R || !d->QN || !d->avar) return SPOCK_EINVAL;
  if (d->nx < 1 || d->nu < 1) return SPOCK_EINVAL;
  if (d->nx > SPOCK_MAX_NX || d->nu > SPOCK_MAX_NU || d->nx + d->nu > MAXD) return SPOCK_EUNSUPPORTED;
  if ((d->x_lo == nullptr) != (d->x_hi == nullptr)) return SPOCK_EINVAL;
  if ((d->u_lo == nullptr) != (d->u_hi == nullptr)) return SPOCK_EINVAL;
  spock_problem* p = new spock_problem();
  int rc = build_tree(p, d->n_nodes, d->anc, d->prob, d->tv ? 1 : 0);
  if (rc) { delete p; return rc; }
  const int n = p->n, n_nl = p->n_nl, n_l = p->n_l, nx = d->nx, nu = d->nu;
  p->nx = nx; p->nu = nu;
  // data checks
  const int full = d->weights_full ? 1 : 0;
  const long long wq = full ? (long long)nx * nx : nx, wr = full ? (long long)nu * nu : nu;
  auto bad = [&](const double* a, long long len) { return a && !finite_arr(a, len); };
  if (bad(d->A, (long long)(n - 1) * nx * nx) || bad(d->B, (long long)(n - 1) * nx * nu) ||
      bad(d->c, (long long)(n - 1) * nx) || bad(d->Q, (long long)(n - 1) * wq) ||
      bad(d->R, (long long)(n - 1) * wr) || bad(d->QN, (long long)n_l * wq) ||
      bad(d->x_lo, (long long)n * nx) || bad(d->x_hi, (long long)n * nx) ||
      bad(d->u_lo, (long long)n_nl * nu) || bad(d->u_hi, (long long)n_nl * nu) ||
      bad(d->u_ball, n_nl) || bad(d->avar, n_nl) || bad(d->q, (long long)(n - 1) * nx) ||
      bad(d->r, (long long)(n - 1) * nu) || bad(d->qN, (long long)n_l * nx)) {
    delete p; return SPOCK_EINVAL;
  }
  // diagonals of the weights (all the preconditioning of Sec. 5.4 uses); full
  // weights must be symmetric with a positive diagonal (the Cholesky factor
  // on the device decides positive definiteness)
  std::vector<double> Qd((size_t)(n - 1) * nx), Rd((size_t)(n - 1) * nu), QNd((size_t)n_l * nx);
  {
    auto take = [&](const double* W, long long nb, int m, std::vector<double>& out) -> bool {
      for (long long b = 0; b < nb; ++b) {
        if (!full) {
          for (int k = 0; k < m; ++k) {
            const double v = W[b * m + k];
            if (v < 0) return false;
            out[(size_t)(b * m + k)] = v;
          }
          continue;
        }
        const double* M = W + b * (long long)m * m;
        double mx = 0.0;
        for (long long e = 0; e < (long long)m * m; ++e) mx = std::max(mx, fabs(M[e]));
        for (int i = 0; i < m; ++i) {
          if (!(M[(size_t)i * m + i] > 0)) return false;
          out[(size_t)(b * m + i)] = M[(size_t)i * m + i];
          for (int j = i + 1; j < m; ++j)
            if (fabs(M[(size_t)i * m + j] - M[(size_t)j * m + i]) > 1e-12 * mx) return false;
        }
      }
      return true;
    };
    if (!take(d->Q, n - 1, nx, Qd) || !take(d->R, n - 1, nu, Rd) || !take(d->QN, n_l, nx, QNd)) {
      delete p; return SPOCK_EINVAL;
    }
    // a linear term needs a positive weight where it is nonzero (Prop. 1, S = I)
    auto lin_ok = [&](const double* w, const std::vector<double>& dg, long long len) {
      if (!w) return true;
      for (long long e = 0; e < len; ++e)
        if (w[e] != 0.0 && !(dg[(size_t)e] > 0)) return false;
      return true;
    };
    if (!lin_ok(d->q, Qd, (long long)(n - 1) * nx) || !lin_ok(d->r, Rd, (long long)(n - 1) * nu) ||
        !lin_ok(d->qN, QNd, (long long)n_l * nx)) {
      delete p; return SPOCK_EINVAL;
    }
  }
  // general rows
  if (d->n_g < 0 || d->n_gN < 0) { delete p; return SPOCK_EINVAL; }
  if (d->n_g > MAXD || d->n_gN > MAXD) { delete p; return SPOCK_EUNSUPPORTED; }
  if (d->n_g > 0) {
    if (!d->Gx || !d->Gu || !d->g_lo || !d->g_hi || bad(d->Gx, (long long)d->n_g * nx) ||
        bad(d->Gu, (long long)d->n_g * nu) || bad(d->g_lo, (long long)n_nl * d->n_g) ||
        bad(d->g_hi, (long long)n_nl * d->n_g)) {
      delete p; return SPOCK_EINVAL;
    }
    for (long long e = 0; e < (long long)n_nl * d->n_g; ++e)
      if (d->g_lo[e] > d->g_hi[e]) { delete p; return SPOCK_EINVAL; }
  }
  if (d->n_gN > 0) {
    if (!d->GN || !d->gN_lo || !d->gN_hi || bad(d->GN, (long long)d->n_gN * nx) ||
        bad(d->gN_lo, (long long)n_l * d->n_gN) || bad(d->gN_hi, (long long)n_l * d->n_gN)) {
      delete p; return SPOCK_EINVAL;
    }
    for (long long e = 0; e < (long long)n_l * d->n_gN; ++e)
      if (d->gN_lo[e] > d->gN_hi[e]) { delete p; return SPOCK_EINVAL; }
  }
  if (!(d->l1 >= 0.0) || !isfinite(d->l1)) { delete p; return SPOCK_EINVAL; }
  p->l1 = d->l1;
  if (d->soft_max) {
    if (d->l1 > 0 || full) { delete p; return SPOCK_EUNSUPPORTED; }
    p->soft = 1;
    p->soft_max.assign(d->soft_max, d->soft_max + nx + nu);
    for (double v : p->soft_max) if (!isfinite(v)) { delete p; return SPOCK_EINVAL; }
  }
  if (d->tv) {
    p->tv = 1;
    p->tvr.assign(d->tv, d->tv + n_nl);
    for (double r : p->tvr) if (!(r >= 0.0) || !isfinite(r)) { delete p; return SPOCK_EINVAL; }
  }
  p->full = full;
  p->has_lin = (d->q || d->r || d->qN) ? 1 : 0;
  p->n_g = d->n_g;
  p->n_gN = d->n_gN;
  for (int i = 0; i < n_nl; ++i) if (d->avar[i] < 0 || d->avar[i] > 1) { delete p; return SPOCK_EINVAL; }
  if (d->x_lo) for (long long e = 0; e < (long long)n * nx; ++e) if (d->x_lo[e] > d->x_hi[e]) { delete p; return SPOCK_EINVAL; }
  if (d->u_lo) for (long long e = 0; e < (long long)n_nl * nu; ++e) if (d->u_lo[e] > d->u_hi[e]) { delete p; return SPOCK_EINVAL; }
  if (d->u_ball) for (int i = 0; i < n_nl; ++i) if (!(d->u_ball[i] >= 0)) { delete p; return SPOCK_EINVAL; }
  p->nbx = d->x_lo ? nx : 0;
  p->nbu = d->u_lo ? nu : 0;
  p->nbox = p->nbx + p->nbu;
  p->has_ball = d->u_ball ? 1 : 0;
  p->n_c = p->nbox + (p->has_ball ? nu : 0) + p->n_g;
  p->n_cN = p->nbx + p->n_gN;
  // layout (Sec. 4.3-4.4)
  p->o_x = 1; p->o_u = p->o_x + (long long)n * nx; p->o_y = p->o_u + (long long)n_nl * nu;
  p->o_tau = p->o_y + p->n_y; p->o_s = p->o_tau + (n - 1); p->nz = p->o_s + (n - 1);
  p->e_y = 0; p->e_s = p->n_y; p->e_c = p->e_s + n_nl; p->e_q = p->e_c + (long long)n_nl * p->n_c;
  p->e_cN = p->e_q + (long long)(n - 1) * (nx + nu + 2);
  p->e_qN = p->e_cN + (long long)n_l * p->n_cN;
  p->neta = p->e_qN + (long long)n_l * (nx + 2);
  // l1 edge costs (Prop. 2): theta, lambda per non-leaf node after s in z, their
  // rows after the leaf cost cones in eta
  p->o_th = p->nz;
  p->o_lam = p->o_th + (p->l1 > 0 ? n_nl : 0);
  p->e_l1 = p->neta;
  if (p->l1 > 0) {
    p->nz = p->o_lam + (long long)n_nl * (nx + nu);
    p->neta = p->e_l1 + (long long)n_nl * (1 + 2 * (nx + nu));
  }
  // soft-constraint costs: sigma, theta per non-leaf node next in z, their rows next in eta
  p->o_sg = p->nz;
  p->o_sth = p->o_sg + (p->soft ? n_nl : 0);
  p->e_sf = p->neta;
  if (p->soft) {
    p->nz = p->o_sth + (long long)n_nl * (nx + nu);
    p->neta = p->e_sf + (long long)n_nl * (3 * (nx + nu) + 2);
  }
  p->nv = p->nz + p->neta;
  p->ldB = pad4(nx + nu); p->ldF = pad4(nx); p->ldP = pad4(nx + nu); p->ldK = pad4(nu);
  p->tw = pick_tw(nx, nu);
  // preconditioning scalings (Sec. 5.4)
  int maxch = 1;
  for (int i = 0; i < n_nl; ++i) maxch = std::max(maxch, p->ch_off[i + 1] - p->ch_off[i]);
  p->maxch = maxch;
  const double chat = sqrt((double)maxch);
  p->Sx.assign(nx, 1.0); p->Su.assign(nu, 1.0); p->SxN.assign(nx, 1.0);
  for (int c = 1; c < n; ++c) {
    for (int k = 0; k < nx; ++k) p->Sx[k] = std::max(p->Sx[k], sqrt(Qd[(size_t)(c - 1) * nx + k]));
    for (int k = 0; k < nu; ++k) p->Su[k] = std::max(p->Su[k], sqrt(Rd[(size_t)(c - 1) * nu + k]));
  }
  for (int j = 0; j < n_l; ++j)
    for (int k = 0; k < nx; ++k) p->SxN[k] = std::max(p->SxN[k], sqrt(QNd[(size_t)j * nx + k]));
  for (int k = 0; k < nx; ++k) p->Sx[k] *= chat;
  for (int k = 0; k < nu; ++k) p->Su[k] *= chat;
  // ||[Gx Sx^-1, Gu Su^-1]||_2 of selection rows: its Gram is diagonal
  {
    double g = 0.0;
    if (p->nbx) for (int k = 0; k < nx; ++k) g = std::max(g, 1.0 / (p->Sx[k] * p->Sx[k]));
    const int nub = (p->nbu ? 1 : 0) + (p->has_ball ? 1 : 0);
    if (nub) for (int k = 0; k < nu; ++k) g = std::max(g, nub / (p->Su[k] * p->Su[k]));
    p->a_con = std::max(1.0, sqrt(g));
    double gN = 0.0;
    if (p->nbx) for (int k = 0; k < nx; ++k) gN = std::max(gN, 1.0 / (p->SxN[k] * p->SxN[k]));
    p->a_conN = std::max(1.0, sqrt(gN));
  }
  // with general rows the Gram of the scaled rows is full: its norm by Jacobi
  std::vector<double> hGg, hGgT, hglo, hghi, hGgN, hGgNT, hgNlo, hgNhi;
  if (p->n_g) {
    const int w = nx + nu, ng = p->n_g;
    const int rows = p->n_c;
    std::vector<double> M((size_t)rows * w, 0.0);
    int r = 0;
    for (int k = 0; k < p->nbx; ++k, ++r) M[(size_t)r * w + k] = 1.0 / p->Sx[k];
    for (int k = 0; k < p->nbu; ++k, ++r) M[(size_t)r * w + nx + k] = 1.0 / p->Su[k];
    if (p->has_ball) for (int k = 0; k < nu; ++k, ++r) M[(size_t)r * w + nx + k] = 1.0 / p->Su[k];
    for (int g = 0; g < ng; ++g, ++r) {
      for (int k = 0; k < nx; ++k) M[(size_t)r * w + k] = d->Gx[(size_t)g * nx + k] / p->Sx[k];
      for (int k = 0; k < nu; ++k) M[(size_t)r * w + nx + k] = d->Gu[(size_t)g * nu + k] / p->Su[k];
    }
    p->a_con = std::max(1.0, mat_norm2(M, rows, w));
    hGg.resize((size_t)ng * w); hGgT.resize((size_t)ng * w);
    for (int g = 0; g < ng; ++g)
      for (int k = 0; k < w; ++k) {
        const double v = M[(size_t)(rows - ng + g) * w + k] / p->a_con;
        hGg[(size_t)g * w + k] = v;
        hGgT[(size_t)k * ng + g] = v;
      }
    hglo.resize((size_t)n_nl * ng); hghi.resize((size_t)n_nl * ng);
    for (long long e = 0; e < (long long)n_nl * ng; ++e) {
      hglo[(size_t)e] = d->g_lo[e] / p->a_con;
      hghi[(size_t)e] = d->g_hi[e] / p->a_con;
    }
  }
  if (p->n_gN) {
    const int ng = p->n_gN, rows = p->n_cN;
    std::vector<double> M((size_t)rows * nx, 0.0);
    int r = 0;
    for (int k = 0; k < p->nbx; ++k, ++r) M[(size_t)r * nx + k] = 1.0 / p->SxN[k];
    for (int g = 0; g < ng; ++g, ++r)
      for (int k = 0; k < nx; ++k) M[(size_t)r * nx + k] = d->GN[(size_t)g * nx + k] / p->SxN[k];
    p->a_conN = std::max(1.0, mat_norm2(M, rows, nx));
    hGgN.resize((size_t)ng * nx); hGgNT.resize((size_t)ng * nx);
    for (int g = 0; g < ng; ++g)
      for (int k = 0; k < nx; ++k) {
        const double v = M[(size_t)(rows - ng + g) * nx + k] / p->a_conN;
        hGgN[(size_t)g * nx + k] = v;
        hGgNT[(size_t)k * ng + g] = v;
      }
    hgNlo.resize((size_t)n_l * ng); hgNhi.resize((size_t)n_l * ng);
    for (long long e = 0; e < (long long)n_l * ng; ++e) {
      hgNlo[(size_t)e] = d->gN_lo[e] / p->a_conN;
      hgNhi[(size_t)e] = d->gN_hi[e] / p->a_conN;
    }
  }
  if (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess) {
    delete p; return SPOCK_EDEVICE;
  }
  DevMem& m = p->mem;
  auto up_i = [&](const std::vector<int>& v) {
    int* q = m.alloc<int>((long long)v.size());
    if (q && !v.empty()) cudaMemcpy(q, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
    return q;
  };
  auto up_d = [&](const double* a, long long len) -> double* {
    if (!a) return nullptr;
    double* q = m.alloc<double>(len);
    if (q) cudaMemcpy(q, a, (size_t)len * sizeof(double), cudaMemcpyHostToDevice);
    return q;
  };
  p->d_anc = up_i(p->anc); p->d_ch_off = up_i(p->ch_off); p->d_yoff = up_i(p->yoff);
  p->d_ynode = up_i(p->ynode); p->d_lvl_off = up_i(p->lvl_off); p->d_seg_top = up_i(p->seg_top);
  p->d_seg_bot = up_i(p->seg_bot); p->d_seg_len = up_i(p->seg_len);
  {
    std::vector<int> ts(n, -1), bs(n, -1);
    for (size_t q = 0; q < p->seg_top.size(); ++q) {
      ts[p->seg_top[q]] = (int)q;
      bs[p->seg_bot[q]] = (int)q;
    }
    p->d_top_seg = up_i(ts);
    p->d_bot_seg = up_i(bs);
  }
  p->d_seg_off = up_i(p->seg_off); p->d_seg_nodes = up_i(p->seg_nodes);
  {
    std::vector<int> info;
    for (size_t q = 0; q < p->seg_top.size(); ++q) {
      const int bot = p->seg_bot[q];
      info.push_back(p->seg_off[q]); info.push_back(p->seg_len[q]);
      info.push_back(p->ch_off[bot]); info.push_back(p->ch_off[bot + 1]);
    }
    p->d_seg_info = reinterpret_cast<int4*>(up_i(info));
  }
  p->d_Sx = up_d(p->Sx.data(), nx); p->d_Su = up_d(p->Su.data(), nu); p->d_SxN = up_d(p->SxN.data(), nx);
  double* d_prob = up_d(d->prob, n);
  double* d_avar = up_d(d->avar, n_nl);
  DevMem tmp;   // setup-only buffers
  double* dA = tmp.alloc<double>((long long)(n - 1) * nx * nx);
  double* dB = tmp.alloc<double>((long long)(n - 1) * nx * nu);
  double* dc = nullptr;
  if (d->c) dc = tmp.alloc<double>((long long)(n - 1) * nx);
  double* dQ = tmp.alloc<double>((long long)(n - 1) * nx);
  double* dR = tmp.alloc<double>((long long)(n - 1) * nu);
  double* dQN = tmp.alloc<double>((long long)n_l * nx);
  double* dxlo = d->x_lo ? tmp.alloc<double>((long long)n * nx) : nullptr;
  double* dxhi = d->x_hi ? tmp.alloc<double>((long long)n * nx) : nullptr;
  double* dulo = d->u_lo ? tmp.alloc<double>((long long)n_nl * nu) : nullptr;
  double* duhi = d->u_hi ? tmp.alloc<double>((long long)n_nl * nu) : nullptr;
  double* dball = d->u_ball ? tmp.alloc<double>(n_nl) : nullptr;
  if (tmp.failed || m.failed) { tmp.free_all(); m.free_all(); delete p; return SPOCK_ENOMEM; }
  cudaMemcpy(dA, d->A, (size_t)(n - 1) * nx * nx * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, d->B, (size_t)(n - 1) * nx * nu * 8, cudaMemcpyHostToDevice);
  if (dc) cudaMemcpy(dc, d->c, (size_t)(n - 1) * nx * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dQ, Qd.data(), (size_t)(n - 1) * nx * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dR, Rd.data(), (size_t)(n - 1) * nu * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dQN, QNd.data(), (size_t)n_l * nx * 8, cudaMemcpyHostToDevice);
  if (dxlo) cudaMemcpy(dxlo, d->x_lo, (size_t)n * nx * 8, cudaMemcpyHostToDevice);
  if (dxhi) cudaMemcpy(dxhi, d->x_hi, (size_t)n * nx * 8, cudaMemcpyHostToDevice);
  if (dulo) cudaMemcpy(dulo, d->u_lo, (size_t)n_nl * nu * 8, cudaMemcpyHostToDevice);
  if (duhi) cudaMemcpy(duhi, d->u_hi, (size_t)n_nl * nu * 8, cudaMemcpyHostToDevice);
  if (dball) cudaMemcpy(dball, d->u_ball, (size_t)n_nl * 8, cudaMemcpyHostToDevice);
  // offline FP64 arrays
  p->d_P = m.alloc<double>((long long)n * nx * nx);
  p->d_K = m.alloc<double>((long long)n_nl * nu * nx);
  p->d_Rt = m.alloc<double>((long long)n_nl * nu * nu);
  p->d_Abar = m.alloc<double>((long long)(n - 1) * nx * nx);
  p->d_x0raw = m.alloc<double>(nx);
  p->d_out_risk = m.alloc<double>(1);
  double* dAt = tmp.alloc<double>((long long)(n - 1) * nx * nx);
  double* dBt = tmp.alloc<double>((long long)(n - 1) * nx * nu);
  double* dLc = tmp.alloc<double>((long long)n_nl * nu * nu);
  double* dLi = tmp.alloc<double>((long long)n_nl * nu * nu);
  double* dRi = tmp.alloc<double>((long long)n_nl * nu * nu);
  double* dKA = tmp.alloc<double>((long long)n_nl * nu * nx);
  double* dBtP = tmp.alloc<double>((long long)n * nu * nx);
  double* dPAb = tmp.alloc<double>((long long)n * nx * nx);
  double* dPcs = tmp.alloc<double>((long long)(n - 1) * nx);
  int* derr = tmp.alloc<int>(1);
  unsigned long long* dnorm = tmp.alloc<unsigned long long>(1);
  rc = alloc_iter<double>(p, p->f64);
  if (!rc) rc = alloc_iter<float>(p, p->f32);
  if (rc || tmp.failed || m.failed) { tmp.free_all(); m.free_all(); delete p; return SPOCK_ENOMEM; }
  double* dct = p->f64.cvec;
  cudaMemset(derr, 0, sizeof(int));
  cudaMemset(dnorm, 0, sizeof(unsigned long long));
  if (!dc) cudaMemset(dct, 0, (size_t)(n - 1) * nx * 8);
  SetupArgs a{};
  a.n = n; a.n_nl = n_nl; a.nx = nx; a.nu = nu; a.nbx = p->nbx; a.nbu = p->nbu; a.has_ball = p->has_ball;
  a.ldB = p->ldB; a.ldF = p->ldF; a.ldP = p->ldP; a.ldK = p->ldK;
  a.a_con = p->a_con; a.a_conN = p->a_conN;
  a.anc = p->d_anc; a.ch_off = p->d_ch_off; a.prob = d_prob;
  a.Sx = p->d_Sx; a.SxN = p->d_SxN; a.Su = p->d_Su;
  a.A = dA; a.B = dB; a.c = dc; a.Qd = dQ; a.Rd = dR; a.QNd = dQN;
  a.xlo = dxlo; a.xhi = dxhi; a.ulo = dulo; a.uhi = duhi; a.uball = dball;
  a.At = dAt; a.Bt = dBt; a.ct = dct;
  a.P = p->d_P; a.K = p->d_K; a.Rt = p->d_Rt; a.Lc = dLc; a.Linv = dLi; a.Rinv = dRi; a.KA = dKA;
  a.BtP = dBtP; a.PAb = dPAb; a.Abar = p->d_Abar; a.err = derr;
  Iter<double>& f = p->f64;
  a.MB = f.MB; a.MF = f.MF; a.MP = f.MP; a.KT = f.KT; a.Pc = dPcs; a.kc = f.kc;
  a.qh = f.qh; a.rh = f.rh; a.qNh = f.qNh; a.gx = f.gx; a.gu = f.gu; a.gN = f.gN;
  a.box_lo = f.box_lo; a.box_hi = f.box_hi; a.boxN_lo = f.boxN_lo; a.boxN_hi = f.boxN_hi; a.ball = f.ball;
  a.ys_block = p->tv ? 0 : 1;
  if (p->soft) {   // 1/s and the scaled lower bounds -s z_max of the soft rows, both precisions
    std::vector<double> w64(nx + nu), l64(nx + nu);
    for (int k = 0; k < nx + nu; ++k) {
      const double sk = (k < nx) ? p->Sx[k] : p->Su[k - nx];
      w64[(size_t)k] = 1.0 / sk;
      l64[(size_t)k] = -sk * p->soft_max[(size_t)k];
    }
    std::vector<float> w32(w64.begin(), w64.end()), l32(l64.begin(), l64.end());
    if (cudaMemcpy(p->f64.smw, w64.data(), w64.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->f64.slo, l64.data(), l64.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->f32.smw, w32.data(), w32.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->f32.slo, l32.data(), l32.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      tmp.free_all(); m.free_all(); delete p; return SPOCK_EDEVICE;
    }
    a.soft_w = p->f64.smw;
  }
  a.xu_shift = (p->l1 > 0) ? 2.0 : 0.0;   // the l1 rows add 2 I to every (x^i, u^i) block of L'L
  cudaStream_t st = 0;
  cudaError_t e = launch_scale_dyn(a, st);
  if (e == cudaSuccess) e = launch_alg1(a, p->stage_off.data(), p->N, st);
  if (e == cudaSuccess) e = launch_build(a, st);
  if (e == cudaSuccess) e = launch_norm_L(a, dnorm, st);
  // full weights: upper Cholesky factors, the cone translations of the
  // linear terms (from the unscaled factors), then the scaled factors
  int* derr2 = tmp.alloc<int>(1);
  if (tmp.failed) { tmp.free_all(); m.free_all(); delete p; return SPOCK_ENOMEM; }
  cudaMemset(derr2, 0, sizeof(int));
  {
    double* dQf = nullptr; double* dRf = nullptr; double* dQNf = nullptr;
    if (full && e == cudaSuccess) {
      dQf = up_tmp(tmp, d->Q, (long long)(n - 1) * nx * nx);
      dRf = up_tmp(tmp, d->R, (long long)(n - 1) * nu * nu);
      dQNf = up_tmp(tmp, d->QN, (long long)n_l * nx * nx);
      if (tmp.failed) { tmp.free_all(); m.free_all(); delete p; return SPOCK_ENOMEM; }
      e = launch_chol_upper(n - 1, nx, dQf, derr2, st);
      if (e == cudaSuccess) e = launch_chol_upper(n - 1, nu, dRf, derr2, st);
      if (e == cudaSuccess) e = launch_chol_upper(n_l, nx, dQNf, derr2, st);
    }
    if (p->has_lin && e == cudaSuccess) {
      double* wq_ = d->q ? tmp.alloc<double>((long long)(n - 1) * nx) : nullptr;
      double* wr_ = d->r ? tmp.alloc<double>((long long)(n - 1) * nu) : nullptr;
      double* wqN = d->qN ? tmp.alloc<double>((long long)n_l * nx) : nullptr;
      double* kap = tmp.alloc<double>(n - 1);
      double* kapN = tmp.alloc<double>(n_l);
      double* dq = up_tmp(tmp, d->q, (long long)(n - 1) * nx);
      double* dr = up_tmp(tmp, d->r, (long long)(n - 1) * nu);
      double* dqN = up_tmp(tmp, d->qN, (long long)n_l * nx);
      if (tmp.failed) { tmp.free_all(); m.free_all(); delete p; return SPOCK_ENOMEM; }
      cudaMemset(kap, 0, (size_t)(n - 1) * 8);
      cudaMemset(kapN, 0, (size_t)n_l * 8);
      if (dq) e = launch_ftinv(n - 1, nx, full, full ? dQf : dQ, dq, wq_, kap, st);
      if (e == cudaSuccess && dr) e = launch_ftinv(n - 1, nu, full, full ? dRf : dR, dr, wr_, kap, st);
      if (e == cudaSuccess && dqN) e = launch_ftinv(n_l, nx, full, full ? dQNf : dQN, dqN, wqN, kapN, st);
      if (e == cudaSuccess) e = launch_translation(n - 1, nx, nu, wq_, wr_, kap, p->f64.acost, st);
      if (e == cudaSuccess) e = launch_translation(n_l, nx, 0, wqN, nullptr, kapN, p->f64.acostN, st);
    }
    if (full && e == cudaSuccess) {
      Iter<double>& f = p->f64;
      e = launch_scale_factor(n - 1, nx, dQf, p->d_Sx, f.FQ, f.FQT, st);
      if (e == cudaSuccess) e = launch_scale_factor(n - 1, nu, dRf, p->d_Su, f.FR, f.FRT, st);
      if (e == cudaSuccess) e = launch_scale_factor(n_l, nx, dQNf, p->d_SxN, f.FN, f.FNT, st);
    }
    if (p->n_g && e == cudaSuccess) {
      Iter<double>& f = p->f64;
      e = cudaMemcpy(f.Gg, hGg.data(), hGg.size() * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(f.GgT, hGgT.data(), hGgT.size() * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(f.gen_lo, hglo.data(), hglo.size() * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(f.gen_hi, hghi.data(), hghi.size() * 8, cudaMemcpyHostToDevice);
    }
    if (p->n_gN && e == cudaSuccess) {
      Iter<double>& f = p->f64;
      e = cudaMemcpy(f.GgN, hGgN.data(), hGgN.size() * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(f.GgNT, hGgNT.data(), hGgNT.size() * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(f.genN_lo, hgNlo.data(), hgNlo.size() * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(f.genN_hi, hgNhi.data(), hgNhi.size() * 8, cudaMemcpyHostToDevice);
    }
  }
  // ||L|| over the blocks of L'L that are not diagonal: (x^i, u^i) of every
  // non-leaf node and x^j of every leaf (the diagonal estimates above are
  // lower bounds of those blocks' largest eigenvalues)
  if ((full || p->n_g || p->n_gN) && e == cudaSuccess) {
    fill_prob<double>(p, p->f64, 1.0);
    e = launch_norm_L_blocks(p->f64.P, dnorm, st);
  }
  if (e == cudaSuccess) e = cudaMemcpy(f.prob, d_prob, (size_t)n * 8, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f.avar, d_avar, (size_t)n_nl * 8, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int herr = 0;
  unsigned long long hnorm = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&hnorm, dnorm, sizeof(hnorm), cudaMemcpyDeviceToHost);
  int herr2 = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr2, derr2, sizeof(int), cudaMemcpyDeviceToHost);
  p->setup_peak = m.bytes + tmp.bytes;   // both sets are at their largest here
  tmp.free_all();
  if (e != cudaSuccess) { m.free_all(); delete p; return SPOCK_EDEVICE; }
  if (herr || herr2) { m.free_all(); delete p; return SPOCK_ENOTPD; }
  double l2;
  memcpy(&l2, &hnorm, sizeof(double));
  if (p->l1 > 0) {
    // the l1 auxiliaries of node i with the tau^c of its m children: L'L on
    // (theta, lambda, tau) is [1 + m l^2/2, -w', -l/2 1'; -w, 2 I + w w', 0;
    // -l/2 1, 0, I/2] (w = 1/s, l = lambda_0). Off span(theta, w, 1) its
    // eigenvalues are 2 and 1/2; on it, the 3 x 3 matrix below.
    double w2 = 0.0;
    for (int k = 0; k < nx; ++k) w2 += 1.0 / (p->Sx[k] * p->Sx[k]);
    for (int k = 0; k < nu; ++k) w2 += 1.0 / (p->Su[k] * p->Su[k]);
    std::vector<int> ms;
    for (int i = 0; i < n_nl; ++i) ms.push_back(p->ch_off[i + 1] - p->ch_off[i]);
    std::sort(ms.begin(), ms.end());
    ms.erase(std::unique(ms.begin(), ms.end()), ms.end());
    l2 = std::max(l2, 2.0);
    for (int m : ms) {
      const double lm = p->l1, sm = sqrt((double)m);
      const double M3[3][3] = {{1.0 + 0.5 * m * lm * lm, -sqrt(w2), -0.5 * lm * sm},
                               {-sqrt(w2), 2.0 + w2, 0.0},
                               {-0.5 * lm * sm, 0.0, 0.5}};
      l2 = std::max(l2, sym3_max_eig(M3));
    }
    std::vector<double> w64(nx + nu);
    std::vector<float> w32(nx + nu);
    for (int k = 0; k < nx + nu; ++k) {
      w64[(size_t)k] = 1.0 / (k < nx ? p->Sx[k] : p->Su[k - nx]);
      w32[(size_t)k] = (float)w64[(size_t)k];
    }
    if (cudaMemcpy(p->f64.l1w, w64.data(), w64.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->f32.l1w, w32.data(), w32.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      m.free_all(); delete p; return SPOCK_EDEVICE;
    }
  }
  if (p->soft) {
    // sigma^i with the tau^c of its m children: [m/2 + 1/2, -1'/2; -1/2, I/2];
    // off the symmetric tau combination 1/2, on it the 2 x 2 below
    for (int i = 0; i < n_nl; ++i) {
      const double m2 = (double)(p->ch_off[i + 1] - p->ch_off[i]);
      const double a = 0.5 * m2 + 0.5, b = 0.5, c = -0.5 * sqrt(m2);
      l2 = std::max(l2, 0.5 * (a + b) + sqrt(0.25 * (a - b) * (a - b) + c * c));
    }
  }
  if (p->tv) {
    // the (y^i, s^i) block of L'L, [I + b b', -b; -b', 1]: 1 + beta/2 + sqrt(beta + beta^2/4),
    // beta = ||b||^2 = 2 ||p||^2 + r^2 + 1 for the total-variation risk
    for (int i = 0; i < n_nl; ++i) {
      double beta = 1.0 + p->tvr[(size_t)i] * p->tvr[(size_t)i];
      for (int c = p->ch_off[i]; c < p->ch_off[i + 1]; ++c) beta += 2.0 * d->prob[c] * d->prob[c];
      l2 = std::max(l2, 1.0 + 0.5 * beta + sqrt(beta + 0.25 * beta * beta));
    }
    std::vector<float> r32(p->tvr.begin(), p->tvr.end());
    if (cudaMemcpy(p->f64.tvr, p->tvr.data(), (size_t)n_nl * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->f32.tvr, r32.data(), (size_t)n_nl * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      m.free_all(); delete p; return SPOCK_EDEVICE;
    }
  }
  p->normL = sqrt(l2);
  p->alpha = 0.99 / p->normL;
  // FP32 copies of the iteration data
  Iter<float>& g = p->f32;
  const long long cnt[] = {(long long)(n - 1) * nx * p->ldB, (long long)(n - 1) * (nx + nu) * p->ldF,
                           (long long)n_nl * nu * p->ldP, (long long)n_nl * nx * p->ldK,
                           (long long)(n - 1) * nx, (long long)n_nl * (nx + nu), (long long)(n - 1) * nx,
                           (long long)(n - 1) * nu, (long long)n_l * nx, nx, nu, nx,
                           (long long)n_nl * std::max(1, p->nbox), (long long)n_nl * std::max(1, p->nbox),
                           (long long)n_l * nx, (long long)n_l * nx, n_nl, n, n_nl};
  const double* src[] = {f.MB, f.MF, f.MP, f.KT, f.cvec, f.kc, f.qh, f.rh, f.qNh, f.gx, f.gu, f.gN,
                         f.box_lo, f.box_hi, f.boxN_lo, f.boxN_hi, f.ball, f.prob, f.avar};
  float* dst[] = {g.MB, g.MF, g.MP, g.KT, g.cvec, g.kc, g.qh, g.rh, g.qNh, g.gx, g.gu, g.gN,
                  g.box_lo, g.box_hi, g.boxN_lo, g.boxN_hi, g.ball, g.prob, g.avar};
  for (int q = 0; q < 19 && e == cudaSuccess; ++q) e = launch_convert_f64_f32(src[q], dst[q], cnt[q], st);
  {
    const long long wW = nx + nu + 2;
    const long long cnt2[] = {(long long)(n - 1) * nx * nx, (long long)(n - 1) * nx * nx,
                              (long long)(n - 1) * nu * nu, (long long)(n - 1) * nu * nu,
                              (long long)n_l * nx * nx, (long long)n_l * nx * nx, (long long)(n - 1) * wW,
                              (long long)n_l * (nx + 2), (long long)p->n_g * (nx + nu), (long long)p->n_g * (nx + nu),
                              (long long)p->n_gN * nx, (long long)p->n_gN * nx, (long long)n_nl * p->n_g,
                              (long long)n_nl * p->n_g, (long long)n_l * p->n_gN, (long long)n_l * p->n_gN};
    const double* src2[] = {f.FQ, f.FQT, f.FR, f.FRT, f.FN, f.FNT, f.acost, f.acostN, f.Gg, f.GgT, f.GgN, f.GgNT,
                            f.gen_lo, f.gen_hi, f.genN_lo, f.genN_hi};
    float* dst2[] = {g.FQ, g.FQT, g.FR, g.FRT, g.FN, g.FNT, g.acost, g.acostN, g.Gg, g.GgT, g.GgN, g.GgNT,
                     g.gen_lo, g.gen_hi, g.genN_lo, g.genN_hi};
    for (int q = 0; q < 16 && e == cudaSuccess; ++q)
      if (src2[q]) e = launch_convert_f64_f32(src2[q], dst2[q], cnt2[q], st);
  }
  // output-column-major factors of the whole-CTA sweeps
  if (e == cudaSuccess && f.cta) {
    e = launch_transpose(f.MB, n - 1, nx, nx + nu, p->ldB, f.ldTB, f.MBt, 64, st);
    if (e == cudaSuccess) e = launch_transpose(f.MF, n - 1, nx + nu, nx, p->ldF, f.ldTF, f.MFt, 64, st);
    if (e == cudaSuccess) e = launch_transpose(f.KT, n_nl, nx, nu, p->ldK, f.ldTK, f.KTt, 64, st);
  }
  if (e == cudaSuccess && g.cta) {
    e = launch_transpose(f.MB, n - 1, nx, nx + nu, p->ldB, g.ldTB, g.MBt, 32, st);
    if (e == cudaSuccess) e = launch_transpose(f.MF, n - 1, nx + nu, nx, p->ldF, g.ldTF, g.MFt, 32, st);
    if (e == cudaSuccess) e = launch_transpose(f.KT, n_nl, nx, nu, p->ldK, g.ldTK, g.KTt, 32, st);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { m.free_all(); delete p; return SPOCK_EDEVICE; }
  cudaMemset(p->d_x0raw, 0, nx * 8);
  cudaMemset(p->f64.x0s, 0, nx * 8);
  cudaMemset(p->f32.x0s, 0, nx * 4);
  fill_prob<double>(p, p->f64, p->alpha);
  fill_prob<float>(p, p->f32, p->alpha);
  *out = p;
  return cuda_err(cudaDeviceSynchronize());
}

void spock_problem_destroy(spock_problem* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  release_bufs(p->f64);
  release_bufs(p->f32);
  if (p->ctr_block) cudaFree(p->ctr_block);
  p->mem.free_all();
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p;
}

int spock_problem_sizes(const spock_problem* p, spock_sizes* o) {
  if (!p || !o) return SPOCK_EINVAL;
  o->n = p->n; o->n_nonleaf = p->n_nl; o->n_leaf = p->n_l; o->N = p->N; o->nx = p->nx; o->nu = p->nu;
  o->n_c = p->n_c; o->n_cN = p->n_cN; o->n_z = p->nz; o->n_eta = p->neta; o->n_v = p->nv;
  const long long words = (long long)(p->n - 1) * (p->nx * p->ldB + (p->nx + p->nu) * p->ldF) +
                          (long long)p->n_nl * (p->nu * p->ldP + p->nx * p->ldK);
  o->factor_bytes_fp64 = words * 8;
  o->factor_bytes_fp32 = words * 4;
  o->solve_bytes_fp64 = solve_buffer_bytes(p, 64);
  o->solve_bytes_fp32 = solve_buffer_bytes(p, 32);
  o->device_bytes = p->mem.bytes + (p->f64.sb_block ? o->solve_bytes_fp64 : 0) +
                    (p->f32.sb_block ? o->solve_bytes_fp32 : 0) + p->ctr_bytes;
  o->device_peak_bytes = std::max(p->setup_peak, o->device_bytes);
  return SPOCK_OK;
}

int spock_problem_alpha(const spock_problem* p, double* alpha, double* normL) {
  if (!p) return SPOCK_EINVAL;
  if (alpha) *alpha = p->alpha;
  if (normL) *normL = p->normL;
  return SPOCK_OK;
}

int spock_problem_set_alpha(spock_problem* p, double alpha) {
  if (!p || !(alpha > 0.0) || !(alpha * p->normL < 1.0)) return SPOCK_EINVAL;
  p->alpha = alpha;
  p->f64.P.alpha = alpha;
  p->f32.P.alpha = (float)alpha;
  return SPOCK_OK;
}

int spock_problem_scalings(const spock_problem* p, double* Sx, double* Su, double* SxN) {
  if (!p) return SPOCK_EINVAL;
  if (Sx) memcpy(Sx, p->Sx.data(), p->nx * 8);
  if (Su) memcpy(Su, p->Su.data(), p->nu * 8);
  if (SxN) memcpy(SxN, p->SxN.data(), p->nx * 8);
  return SPOCK_OK;
}

int spock_problem_factors(const spock_problem* p, double* P, double* K, double* Rt, double* Abar) {
  if (!p) return SPOCK_EINVAL;
  cudaError_t e = cudaSuccess;
  if (P) e = cudaMemcpy(P, p->d_P, (size_t)p->n * p->nx * p->nx * 8, cudaMemcpyDeviceToHost);
  if (K && e == cudaSuccess) e = cudaMemcpy(K, p->d_K, (size_t)p->n_nl * p->nu * p->nx * 8, cudaMemcpyDeviceToHost);
  if (Rt && e == cudaSuccess) e = cudaMemcpy(Rt, p->d_Rt, (size_t)p->n_nl * p->nu * p->nu * 8, cudaMemcpyDeviceToHost);
  if (Abar && e == cudaSuccess) e = cudaMemcpy(Abar, p->d_Abar, (size_t)(p->n - 1) * p->nx * p->nx * 8, cudaMemcpyDeviceToHost);
  return cuda_err(e);
}

static int set_x0_dev(spock_problem* p, const double* x0_dev, cudaStream_t st) {
  k_scale_x0<<<1, 128, 0, st>>>(p->nx, x0_dev, p->d_Sx, p->f64.x0s, p->f32.x0s);
  return cuda_err(cudaGetLastError());
}

int spock_problem_set_x0(spock_problem* p, const double* x0) {
  if (!p || !x0) return SPOCK_EINVAL;
  if (!finite_arr(x0, p->nx)) return SPOCK_EINVAL;
  if (cudaMemcpy(p->d_x0raw, x0, p->nx * 8, cudaMemcpyHostToDevice) != cudaSuccess) return SPOCK_EDEVICE;
  int rc = set_x0_dev(p, p->d_x0raw, 0);
  if (rc) return rc;
  return cuda_err(cudaDeviceSynchronize());
}

int spock_op_T(spock_problem* p, int precision, const void* v_in, void* v_out, double* stats,
               void* stream) {
  if (!p || !v_in || !v_out || (precision != 32 && precision != 64)) return SPOCK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  SolveOpts so{1e300, 0, 1, 2, 1e-10};
  SolveCtl h{};
  int rc;
  if (precision == 64) {
    rc = ensure_bufs(p, p->f64);
    if (rc) return rc;
    Iter<double> it = p->f64;               // shallow copy with the caller's vectors
    it.sb.V = (double*)v_in;
    it.sb.TV = (double*)v_out;
    it.have_bufs = true;
    rc = run_solver<double>(p, it, so, st, &h, nullptr);
  } else {
    rc = ensure_bufs(p, p->f32);
    if (rc) return rc;
    Iter<float> it = p->f32;
    it.sb.V = (float*)v_in;
    it.sb.TV = (float*)v_out;
    it.have_bufs = true;
    rc = run_solver<float>(p, it, so, st, &h, nullptr);
  }
  if (rc) return rc;
  if (stats)
    for (int k = 0; k < 8; ++k) stats[k] = h.stats[k];
  return SPOCK_OK;
}

int spock_op_T_centred(spock_problem* p, const double* c, const float* delta, float* out, double* stats,
                       void* stream) {
  if (!p || !c || !delta || !out) return SPOCK_EINVAL;
  return spock::op_T_centred(p, c, delta, out, stats, (cudaStream_t)stream);
}

int spock_op_L(spock_problem* p, int precision, const void* z, void* eta, void* stream) {
  if (!p || !z || !eta) return SPOCK_EINVAL;
  cudaError_t e;
  if (precision == 64) e = launch_apply_L<double>(p->f64.P, p->d_ynode, (const double*)z, (double*)eta, (cudaStream_t)stream);
  else if (precision == 32) e = launch_apply_L<float>(p->f32.P, p->d_ynode, (const float*)z, (float*)eta, (cudaStream_t)stream);
  else return SPOCK_EINVAL;
  if (e != cudaSuccess) return SPOCK_EDEVICE;
  return cuda_err(cudaStreamSynchronize((cudaStream_t)stream));
}

int spock_op_Lt(spock_problem* p, int precision, const void* eta, void* z, void* stream) {
  if (!p || !z || !eta) return SPOCK_EINVAL;
  cudaError_t e;
  if (precision == 64) e = launch_apply_Lt<double>(p->f64.P, p->d_ynode, (const double*)eta, (double*)z, (cudaStream_t)stream);
  else if (precision == 32) e = launch_apply_Lt<float>(p->f32.P, p->d_ynode, (const float*)eta, (float*)z, (cudaStream_t)stream);
  else return SPOCK_EINVAL;
  if (e != cudaSuccess) return SPOCK_EDEVICE;
  return cuda_err(cudaStreamSynchronize((cudaStream_t)stream));
}

int spock_solve_device(spock_problem* p, const double* x0, const spock_solve_opts* opts,
                       double* x_out, double* u_out, void* stream, spock_info* info) {
  if (!p || !x0) return SPOCK_EINVAL;
  spock_solve_opts o;
  if (opts) o = *opts;
  else spock_solve_opts_default(&o);
  if ((o.precision != 32 && o.precision != 64) || !(o.tol >= 0) || o.max_iters < 0 ||
      o.max_backtracks < 1 || o.method < 0 || o.method > 1 || o.aa_mode < 0 || o.aa_mode > 1 ||
      !(o.recentre >= 0.0 && o.recentre < 1.0))
    return SPOCK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = set_x0_dev(p, x0, st);
  if (rc) return rc;
  SolveOpts so{};
  so.tol = o.tol; so.max_iters = o.max_iters; so.max_backtracks = o.max_backtracks;
  so.method = o.method; so.rank_tol = (o.precision == 64) ? 1e-10 : 1e-5;
  so.aa_qr = o.aa_mode == 1 ? 1 : 0;
  SolveCtl h{};
  float ms = 0.f;
  double res64 = -1.0;
  double diag6[6];
  bool have_diag = false;
  int n_ctr = 0;
  double kern_ms = -1.0;
  const long long nv = p->nv;
  if (o.precision == 64) {
    rc = ensure_bufs(p, p->f64);
    if (rc) return rc;
    if (!o.warm_start && cudaMemsetAsync(p->f64.sb.V, 0, nv * 8, st) != cudaSuccess) return SPOCK_EDEVICE;
    rc = run_solver<double>(p, p->f64, so, st, &h, &ms);
    if (rc) return rc;
    // keep the final iterate in V for warm starts
    double* fv = buf_index(p->f64.sb, h.final_v);
    if (fv != p->f64.sb.V) cudaMemcpyAsync(p->f64.sb.V, fv, nv * 8, cudaMemcpyDeviceToDevice, st);
    const double* z = buf_index(p->f64.sb, h.final_tv);
    double* tz = p->f64.sb.PSI;   // T(v) copy (PSI is free after the solve)
    cudaMemcpyAsync(tz, z, nv * 8, cudaMemcpyDeviceToDevice, st);
    k_unscale<double><<<64, 256, 0, st>>>(p->n, p->n_nl, p->nx, p->nu, p->o_x, p->o_u, tz, p->d_Sx,
                                         p->d_SxN, p->d_Su, x_out, u_out, p->d_out_risk);
    res64 = h.res_inf;
    // FP64 exit check of (v, T(v)) as they stand (Sec. 5.3)
    rc = diag_run(p, p->f64.sb.V, z, st, diag6);
    if (rc) return rc;
    have_diag = true;
  } else if (o.recentre > 0.0) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    rc = solve_centred(p, o, so, st, x_out, u_out, h, res64, diag6, n_ctr, kern_ms);
    cudaEventRecord(e1, st);
    if (!rc && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    have_diag = true;
  } else {
    rc = ensure_bufs(p, p->f32);
    if (rc) return rc;
    if (!o.warm_start && cudaMemsetAsync(p->f32.sb.V, 0, nv * 4, st) != cudaSuccess) return SPOCK_EDEVICE;
    rc = run_solver<float>(p, p->f32, so, st, &h, &ms);
    if (rc) return rc;
    float* fv = buf_index(p->f32.sb, h.final_v);
    if (fv != p->f32.sb.V) cudaMemcpyAsync(p->f32.sb.V, fv, nv * 4, cudaMemcpyDeviceToDevice, st);
    const float* z = buf_index(p->f32.sb, h.final_tv);
    float* tz = p->f32.sb.PSI;
    cudaMemcpyAsync(tz, z, nv * 4, cudaMemcpyDeviceToDevice, st);
    k_unscale<float><<<64, 256, 0, st>>>(p->n, p->n_nl, p->nx, p->nu, p->o_x, p->o_u, tz, p->d_Sx,
                                        p->d_SxN, p->d_Su, x_out, u_out, p->d_out_risk);
    res64 = h.res_inf;
    if (o.fp64_check) {
      // FP64 exit check of the FP32 iterate: one FP64 evaluation of T, the
      // residual, xi1, xi2, infeasibility and gap (Sec. 5.3)
      double out7[7];
      rc = check_fp64(p, 32, p->f32.sb.V, st, out7);
      if (rc) return rc;
      res64 = out7[0];
      for (int q = 0; q < 6; ++q) diag6[q] = out7[1 + q];
      have_diag = true;
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPOCK_EDEVICE;
  double risk = 0.0;
  cudaMemcpy(&risk, p->d_out_risk, 8, cudaMemcpyDeviceToHost);
  if (info) {
    info->status = h.status == 0 ? SPOCK_OK : SPOCK_MAXITER;
    info->iters = h.iters; info->n_T = h.n_T; info->n_K0 = h.n_K0; info->n_K1 = h.n_K1;
    info->n_K2 = h.n_K2; info->n_fallback = h.n_fb; info->n_backtracks = h.n_bt;
    info->res_inf = h.res_inf; info->res_inf_fp64 = res64; info->risk = risk;
    info->device_ms = ms;
    for (int q = 0; q < 7; ++q) info->phase_ms[q] = 1e-6 * (double)h.prof[q];
    for (int q = 0; q < 8; ++q) info->counters[q] = (double)h.prof[8 + q];
    info->xi1 = have_diag ? diag6[0] : NAN;
    info->xi2 = have_diag ? diag6[1] : NAN;
    info->infeas = have_diag ? diag6[2] : NAN;
    info->gap = have_diag ? diag6[3] : NAN;
    info->n_recentre = n_ctr;
    info->kernel_ms = kern_ms >= 0.0 ? kern_ms : ms;
  }
  return h.status == 0 ? SPOCK_OK : SPOCK_MAXITER;
}

int spock_solve(spock_problem* p, const double* x0, const spock_solve_opts* opts, double* x_out,
                double* u_out, double* risk, spock_info* info) {
  if (!p || !x0) return SPOCK_EINVAL;
  if (!finite_arr(x0, p->nx)) return SPOCK_EINVAL;
  double* dx = nullptr;
  double* du = nullptr;
  const size_t bx = (size_t)p->n * p->nx * 8, bu = (size_t)p->n_nl * p->nu * 8;
  if (x_out && cudaMalloc(&dx, bx) != cudaSuccess) return SPOCK_ENOMEM;
  if (u_out && cudaMalloc(&du, bu) != cudaSuccess) { cudaFree(dx); return SPOCK_ENOMEM; }
  cudaMemcpy(p->d_x0raw, x0, p->nx * 8, cudaMemcpyHostToDevice);
  spock_info inf{};
  int rc = spock_solve_device(p, p->d_x0raw, opts, dx, du, nullptr, &inf);
  if (rc >= 0) {
    if (x_out) cudaMemcpy(x_out, dx, bx, cudaMemcpyDeviceToHost);
    if (u_out) cudaMemcpy(u_out, du, bu, cudaMemcpyDeviceToHost);
    if (risk) *risk = inf.risk;
    if (info) *info = inf;
  }
  if (dx) cudaFree(dx);
  if (du) cudaFree(du);
  return rc;
}

int spock_check(spock_problem* p, int precision, const void* v, void* stream, spock_check_info* out) {
  if (!p || !v || !out || (precision != 32 && precision != 64)) return SPOCK_EINVAL;
  double o7[7];
  const int rc = check_fp64(p, precision, v, (cudaStream_t)stream, o7);
  if (rc) return rc;
  out->res_inf = o7[0]; out->xi1 = o7[1]; out->xi2 = o7[2]; out->infeas = o7[3]; out->gap = o7[4];
  out->eta_Lz = o7[5]; out->support = o7[6];
  return SPOCK_OK;
}

int spock_get_iterate(spock_problem* p, int precision, void* v_out, void* stream) {
  if (!p || !v_out) return SPOCK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == 64) {
    int rc = ensure_bufs(p, p->f64);
    if (rc) return rc;
    return cuda_err(cudaMemcpyAsync(v_out, p->f64.sb.V, p->nv * 8, cudaMemcpyDeviceToDevice, st));
  }
  if (precision == 32) {
    int rc = ensure_bufs(p, p->f32);
    if (rc) return rc;
    return cuda_err(cudaMemcpyAsync(v_out, p->f32.sb.V, p->nv * 4, cudaMemcpyDeviceToDevice, st));
  }
  return SPOCK_EINVAL;
}

int spock_set_iterate(spock_problem* p, int precision, const void* v_in, void* stream) {
  if (!p || !v_in) return SPOCK_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == 64) {
    int rc = ensure_bufs(p, p->f64);
    if (rc) return rc;
    return cuda_err(cudaMemcpyAsync(p->f64.sb.V, v_in, p->nv * 8, cudaMemcpyDeviceToDevice, st));
  }
  if (precision == 32) {
    int rc = ensure_bufs(p, p->f32);
    if (rc) return rc;
    return cuda_err(cudaMemcpyAsync(p->f32.sb.V, v_in, p->nv * 4, cudaMemcpyDeviceToDevice, st));
  }
  return SPOCK_EINVAL;
}

}  // extern "C"
