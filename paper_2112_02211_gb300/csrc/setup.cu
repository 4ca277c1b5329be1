// Setup of the HPS operators on the device (per medium, not per iteration).
//
// Per leaf (Sec. 2.1, eq. (leaf)): assemble the dense leaf matrix
//   A = [ -(D_x^2 + D_y^2 + D_z^2) - C ]   interior rows
//       [  N + i eta I(I_b, :)          ]   face rows (eq. (flux), F)
// augmented with identity columns, and eliminate it with partial pivoting
// (FP64).  Eliminating the last n_b pivots Gauss-Jordan style turns the
// bottom-right block of U into I, so the boundary rows of the augmented part
// are (A^{-1})_{b,:} directly:
//   R_C = I - 2 i eta (A^{-1})_bb,   H_C = -2 i eta (A^{-1})_bi,
// which follows from g = G u = F u - 2 i eta u_b (eq. (G)).  The face data is
// then moved to Gauss points: R = P R_C P^{-1}, H = P H_C, P = blockdiag(Q (x) Q).
//
// Preconditioner (Sec. 4, Sec. 4.1): the same leaf maps with C replaced by
// lambda^tau = (max + min)/2 of C over the leaf (homogenized, R~).  For every
// cluster of leaves, J_c = I + Pi_c R~ ordered (external, internal) is
// [[I, 0], [B, I + D]], so J_c^{-1} r needs K_c = (I + D)^{-1} (dense, inverted
// here by the same elimination kernel) and the blocks B^beta of R~ (internal
// rows, external columns of each leaf).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <type_traits>

#include "common.cuh"
#include "hps_internal.h"

namespace hps {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxP = 16;

// ---------------------------------------------------------------------------
// 1D tables: Chebyshev extreme points, differentiation matrices (Sec. 2.1),
// Gauss-Legendre points by Newton's method on the Legendre recurrence, the
// Lagrange interpolation Q from interior Chebyshev points to Gauss points and
// its inverse.  One thread; p <= 16.
// ---------------------------------------------------------------------------
__global__ void tables_kernel(double* T, TableLayout tl, double hx, double hy, double hz) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int p = tl.p, q = tl.q;
  double* x = T + tl.x;
  for (int j = 0; j < p; ++j) x[j] = -cos(kPi * (double)j / (double)(p - 1));
  double Dr[kMaxP * kMaxP];
  for (int i = 0; i < p; ++i) {
    double ci = (i == 0 || i == p - 1) ? 2.0 : 1.0;
    double rs = 0.0;
    for (int j = 0; j < p; ++j) {
      if (j == i) continue;
      double cj = (j == 0 || j == p - 1) ? 2.0 : 1.0;
      double sg = ((i + j) & 1) ? -1.0 : 1.0;
      double v = (ci / cj) * sg / (x[i] - x[j]);
      Dr[i * p + j] = v;
      rs += v;
    }
    Dr[i * p + i] = -rs;
  }
  const double hh[3] = {hx, hy, hz};
  for (int a = 0; a < 3; ++a) {
    double* D = T + tl.D + a * p * p;
    double s = 2.0 / hh[a];
    for (int i = 0; i < p * p; ++i) D[i] = s * Dr[i];
    double* D2 = T + tl.D2 + a * p * p;
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) {
        double acc = 0.0;
        for (int m = 0; m < p; ++m) acc += D[i * p + m] * D[m * p + j];
        D2[i * p + j] = acc;
      }
  }
  // Gauss-Legendre nodes: Newton iteration from the standard cosine guesses.
  double* xg = T + tl.xg;
  double* wg = T + tl.wg;
  for (int i = 0; i < q; ++i) {
    double z = cos(kPi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < q; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < q; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
    }
    xg[q - 1 - i] = z;  // guesses run from +1 downwards; store ascending
    wg[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  // Q[a][j]: Lagrange basis j of the interior Chebyshev points x[1..p-2] at xg[a].
  double* Q = T + tl.Q;
  for (int a = 0; a < q; ++a)
    for (int j = 0; j < q; ++j) {
      double v = 1.0;
      for (int m = 0; m < q; ++m)
        if (m != j) v *= (xg[a] - x[m + 1]) / (x[j + 1] - x[m + 1]);
      Q[a * q + j] = v;
    }
  // Qi = Q^{-1} by Gauss-Jordan with partial pivoting.
  double Wm[kMaxP * 2 * kMaxP];
  const int w2 = 2 * q;
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < w2; ++j) Wm[i * w2 + j] = (j < q) ? Q[i * q + j] : (j - q == i ? 1.0 : 0.0);
  for (int k = 0; k < q; ++k) {
    int piv = k;
    for (int r = k + 1; r < q; ++r)
      if (fabs(Wm[r * w2 + k]) > fabs(Wm[piv * w2 + k])) piv = r;
    if (piv != k)
      for (int j = 0; j < w2; ++j) {
        double t = Wm[k * w2 + j];
        Wm[k * w2 + j] = Wm[piv * w2 + j];
        Wm[piv * w2 + j] = t;
      }
    double inv = 1.0 / Wm[k * w2 + k];
    for (int j = 0; j < w2; ++j) Wm[k * w2 + j] *= inv;
    for (int r = 0; r < q; ++r) {
      if (r == k) continue;
      double m = Wm[r * w2 + k];
      if (m == 0.0) continue;
      for (int j = 0; j < w2; ++j) Wm[r * w2 + j] -= m * Wm[k * w2 + j];
    }
  }
  double* Qi = T + tl.Qi;
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) Qi[i * q + j] = Wm[i * w2 + q + j];
}

// ---------------------------------------------------------------------------
// Node coordinates.
// ---------------------------------------------------------------------------
__global__ void nodes_kernel(const double* T, TableLayout tl, int nx, int ny, int nz, double* xi,
                             double* xf, double* xc) {
  const int p = tl.p, q = tl.q, n1 = p - 2;
  const long long nl = (long long)nx * ny * nz;
  const long long ni = (long long)n1 * n1 * n1, nb = 6LL * q * q;
  const double h[3] = {1.0 / nx, 1.0 / ny, 1.0 / nz};
  const double* x = T + tl.x;
  const double* xg = T + tl.xg;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = tid; t < nl * (ni > nb ? ni : nb); t += stride) {
    long long leaf = t / (ni > nb ? ni : nb);
    long long r = t % (ni > nb ? ni : nb);
    int ix = (int)(leaf % nx), iy = (int)((leaf / nx) % ny), iz = (int)(leaf / ((long long)nx * ny));
    double c[3] = {ix * h[0], iy * h[1], iz * h[2]};
    if (xi && r < ni) {
      int i = (int)(r % n1) + 1, j = (int)((r / n1) % n1) + 1, k = (int)(r / ((long long)n1 * n1)) + 1;
      double* o = xi + 3 * (leaf * ni + r);
      o[0] = c[0] + 0.5 * h[0] * (x[i] + 1.0);
      o[1] = c[1] + 0.5 * h[1] * (x[j] + 1.0);
      o[2] = c[2] + 0.5 * h[2] * (x[k] + 1.0);
    }
    if (xf && r < nb) {
      int face = (int)(r / (q * q)), jj = (int)(r % (q * q));
      int j1 = jj % q, j2 = jj / q;
      int axis = face >> 1;
      int a0 = (axis == 0) ? 1 : 0, a1 = (axis == 2) ? 1 : 2;
      double* o = xf + 3 * (leaf * nb + r);
      o[axis] = c[axis] + ((face & 1) ? h[axis] : 0.0);
      o[a0] = c[a0] + 0.5 * h[a0] * (xg[j1] + 1.0);
      o[a1] = c[a1] + 0.5 * h[a1] * (xg[j2] + 1.0);
    }
    if (xc && r < nb) {  // Chebyshev face nodes (q == n1): first in-face axis fastest
      int face = (int)(r / (q * q)), jj = (int)(r % (q * q));
      int a = jj % q + 1, bb = jj / q + 1;
      int axis = face >> 1;
      int a0 = (axis == 0) ? 1 : 0, a1 = (axis == 2) ? 1 : 2;
      double* o = xc + 3 * (leaf * nb + r);
      o[axis] = c[axis] + ((face & 1) ? h[axis] : 0.0);
      o[a0] = c[a0] + 0.5 * h[a0] * (x[a] + 1.0);
      o[a1] = c[a1] + 0.5 * h[a1] * (x[bb] + 1.0);
    }
  }
}

// Local index of grid node (i, j, k), 0 <= i,j,k < p, not on an edge/corner.
__device__ __forceinline__ int gidx(int i, int j, int k, int p, int n1, int ni) {
  const int last = p - 1;
  const bool bi = (i == 0 || i == last), bj = (j == 0 || j == last), bk = (k == 0 || k == last);
  if (!bi && !bj && !bk) return (i - 1) + n1 * ((j - 1) + n1 * (k - 1));
  int face, a, b;
  if (bi) { face = (i == 0) ? 0 : 1; a = j; b = k; }
  else if (bj) { face = (j == 0) ? 2 : 3; a = i; b = k; }
  else { face = (k == 0) ? 4 : 5; a = i; b = j; }
  return ni + face * n1 * n1 + (a - 1) + n1 * (b - 1);
}

// ---------------------------------------------------------------------------
// Leaf matrix assembly into a zeroed row-major workspace (one thread per row).
// Columns [0, n): A; with ecols >= 1 also [n, n+nb): e_{boundary}; with
// ecols == 2 also [n+nb, n+nb+ni): e_{interior}.  Interior rows take C from cdiag, or the leaf constant
// lam[leaf] for the homogenized operator.
// ---------------------------------------------------------------------------
template <class T>
__global__ void assemble_kernel(T* W, long long wstride, int ld, const int* leaf_ids, int leaf0,
                                int nbatch, const double* tab, TableLayout tl, double eta,
                                const double2* cdiag, const double2* lam, int ecols) {
  const int p = tl.p, n1 = p - 2, ni = n1 * n1 * n1, nb = 6 * n1 * n1, n = ni + nb;
  const int b = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbatch || r >= n) return;
  const int leaf = leaf_ids ? leaf_ids[b] : leaf0 + b;
  T* row = W + (long long)b * wstride + (long long)r * ld;
  const double* D = tab + tl.D;
  const double* D2 = tab + tl.D2;
  if (r < ni) {
    const int i = r % n1 + 1, j = (r / n1) % n1 + 1, k = r / (n1 * n1) + 1;
    for (int m = 0; m < p; ++m) {
      row[gidx(m, j, k, p, n1, ni)].x -= D2[0 * p * p + i * p + m];
      row[gidx(i, m, k, p, n1, ni)].x -= D2[1 * p * p + j * p + m];
      row[gidx(i, j, m, p, n1, ni)].x -= D2[2 * p * p + k * p + m];
    }
    const double2 c = lam ? lam[leaf] : cdiag[(long long)leaf * ni + r];
    row[r].x -= c.x;
    row[r].y -= c.y;
    if (ecols == 2) row[n + nb + r].x = 1.0;
  } else {
    const int jb = r - ni;
    const int face = jb / (n1 * n1), rem = jb % (n1 * n1);
    const int a = rem % n1 + 1, bb = rem / n1 + 1;
    const int axis = face >> 1;
    const int e = (face & 1) ? p - 1 : 0;
    const double sg = (face & 1) ? 1.0 : -1.0;
    int pt[3];
    pt[axis] = e;
    pt[axis == 0 ? 1 : 0] = a;
    pt[axis == 2 ? 1 : 2] = bb;
    for (int m = 0; m < p; ++m) {
      int q3[3] = {pt[0], pt[1], pt[2]};
      q3[axis] = m;
      row[gidx(q3[0], q3[1], q3[2], p, n1, ni)].x += sg * D[axis * p * p + e * p + m];
    }
    row[r].y += eta;
    if (ecols >= 1) row[n + jb].x = 1.0;
  }
}

// ---------------------------------------------------------------------------
// Batched elimination with partial pivoting, one CTA per matrix (row-major,
// n rows, ncols >= n columns).  Pivots k >= gj0 also eliminate the rows
// [gj0, k) above them, so on exit rows [gj0, n) of columns [n, ncols) hold
// the corresponding rows of A^{-1} E.  A zero pivot sets *status = 1.
// ---------------------------------------------------------------------------
// v -= m u (complex), the elimination's one update
template <class T>
__device__ __forceinline__ void gj_update(T& v, const T m, const T u) {
  v.x -= m.x * u.x - m.y * u.y;
  v.y -= m.x * u.y + m.y * u.x;
}

template <class T, int NT>
__global__ void __launch_bounds__(NT) gj_kernel(T* W, long long wstride, int ld, int n, int ncols,
                                                int gj0, int nbatch, int* status) {
  extern __shared__ __align__(16) unsigned char gj_smem[];
  T* prow = reinterpret_cast<T*>(gj_smem);
  __shared__ double sval[NT / 32];
  __shared__ int sidx[NT / 32];
  __shared__ int piv_s;
  if ((int)blockIdx.x >= nbatch) return;
  T* M = W + (long long)blockIdx.x * wstride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = n;
    for (int r = k + tid; r < n; r += NT) {
      const T v = M[(long long)r * ld + k];
      double a = fabs(v.x) + fabs(v.y);
      if (a > best) { best = a; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { sval[warp] = best; sidx[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      best = (lane < NT / 32) ? sval[lane] : -1.0;
      bi = (lane < NT / 32) ? sidx[lane] : n;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        if (!(best > 0.0) || bi >= n) {
          atomicExch(status, 1);
          bi = k;
        }
        piv_s = bi;
      }
    }
    __syncthreads();
    const int piv = piv_s;
    const T pv = M[(long long)piv * ld + k];
    const T inv = (pv.x == 0 && pv.y == 0) ? czero<T>() : cinv(pv);
    for (int c = k + tid; c < ncols; c += NT) {
      T a = M[(long long)piv * ld + c];
      if (piv != k) M[(long long)piv * ld + c] = M[(long long)k * ld + c];
      a = cmul(a, inv);
      prow[c] = a;
      M[(long long)k * ld + c] = a;
    }
    __syncthreads();
    const int lo = (k >= gj0) ? gj0 : k + 1;
    for (int r = lo + warp; r < n; r += NT / 32) {
      if (r == k) continue;
      T* Mr = M + (long long)r * ld;
      const T m = Mr[k];
      if (m.x == 0 && m.y == 0) continue;
      // four loads in flight per lane; every element gets the same update as one at a time
      int c = k + 1 + lane;
      for (; c + 96 < ncols; c += 128) {
        T v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = Mr[c + 32 * e];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          gj_update(v[e], m, prow[c + 32 * e]);
          Mr[c + 32 * e] = v[e];
        }
      }
      for (; c < ncols; c += 32) {
        T v = Mr[c];
        gj_update(v, m, prow[c]);
        Mr[c] = v;
      }
    }
    __syncthreads();
  }
}

// R_C = I - 2 i eta X_bb and (optionally) H_C = -2 i eta X_bi from the
// eliminated workspace, written to per-leaf storage with leading dims ldr/ldh.
template <class T>
__global__ void extract_kernel(const T* W, long long wstride, int ld, int n, int ni, int nb,
                               double eta, int nbatch, T* R, long long rstride, int ldr,
                               T* H, long long hstride, int ldh) {
  const int b = blockIdx.y;
  if (b >= nbatch) return;
  const int ncols_out = nb + (H ? ni : 0);
  const T* Wb = W + (long long)b * wstride;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nb * ncols_out;
       t += (long long)gridDim.x * blockDim.x) {
    const int jb = (int)(t / ncols_out), c = (int)(t % ncols_out);
    const double2 v = cvt<double2>(Wb[(long long)(ni + jb) * ld + n + c]);
    // -2 i eta (v.x + i v.y) = 2 eta v.y - 2 i eta v.x
    double2 o = make_double2(2.0 * eta * v.y, -2.0 * eta * v.x);
    if (c < nb) {
      if (c == jb) o.x += 1.0;
      R[(long long)b * rstride + (long long)jb * ldr + c] = cvt<T>(o);
    } else {
      H[(long long)b * hstride + (long long)jb * ldh + (c - nb)] = cvt<T>(o);
    }
  }
}

// In-place S <- A S A^T on q x q segments of a batch of matrices.
// mode 0: segment (row r, block f) = M[r][f q^2 + j]; mode 1: (col c, block f)
// = M[f q^2 + j][c].  A = Q (trans = 0) or Q^{-T} (trans = 1; from Qi).
template <class T>
__global__ void seg_kron_kernel(T* M, long long mstride, int ld, int nrows, int ncols, int nbatch,
                                const double* tab, TableLayout tl, int trans, int mode) {
  extern __shared__ __align__(16) unsigned char sk_smem[];
  T* sm = reinterpret_cast<T*>(sk_smem);
  using R_ = typename Real<T>::type;
  const int q = tl.q, q2 = q * q;
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* S = sm + warp * 2 * q2;
  T* T1 = S + q2;
  const double* Am = tab + (trans ? tl.Qi : tl.Q);
  const long long nseg_per = (mode == 0) ? (long long)nrows * (ncols / q2) : (long long)ncols * (nrows / q2);
  const long long nseg = nseg_per * nbatch;
  for (long long s = (long long)blockIdx.x * warps + warp; s < nseg; s += (long long)gridDim.x * warps) {
    const long long b = s / nseg_per, sl = s % nseg_per;
    T* base = M + b * mstride;
    long long off;
    long long es;
    if (mode == 0) {
      const int nf = ncols / q2;
      const long long r = sl / nf;
      const int f = (int)(sl % nf);
      off = r * ld + (long long)f * q2;
      es = 1;
    } else {
      const long long c = sl % ncols;
      const int f = (int)(sl / ncols);
      off = (long long)f * q2 * ld + c;
      es = ld;
    }
    for (int j = lane; j < q2; j += 32) S[j] = base[off + j * es];
    __syncwarp();
    // T1[j2][a] = sum_j1 S[j2][j1] A(a, j1)
    for (int e = lane; e < q2; e += 32) {
      const int j2 = e / q, a = e % q;
      T acc = czero<T>();
      for (int j1 = 0; j1 < q; ++j1) {
        const R_ av = (R_)(trans ? Am[j1 * q + a] : Am[a * q + j1]);
        acc.x += S[j2 * q + j1].x * av;
        acc.y += S[j2 * q + j1].y * av;
      }
      T1[e] = acc;
    }
    __syncwarp();
    // out[bq][a] = sum_j2 A(bq, j2) T1[j2][a]
    for (int e = lane; e < q2; e += 32) {
      const int bq = e / q, a = e % q;
      T acc = czero<T>();
      for (int j2 = 0; j2 < q; ++j2) {
        const R_ av = (R_)(trans ? Am[j2 * q + bq] : Am[bq * q + j2]);
        acc.x += av * T1[j2 * q + a].x;
        acc.y += av * T1[j2 * q + a].y;
      }
      base[off + e * es] = acc;
    }
    __syncwarp();
  }
}

__global__ void cast_kernel(const double2* in, float2* out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void cdiag_kernel(const double2* b, double kappa, long long count, double2* c) {
  const double k2 = kappa * kappa;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    c[i] = make_double2(k2 * (1.0 - b[i].x), -k2 * b[i].y);
}

// lambda^tau = (max + min)/2 of C over the leaf, real and imaginary parts separately.
__global__ void lambda_kernel(const double2* c, int ni, double2* lam) {
  const int leaf = blockIdx.x;
  double mxr = -1e300, mnr = 1e300, mxi = -1e300, mni = 1e300;
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    double2 v = c[(long long)leaf * ni + i];
    mxr = fmax(mxr, v.x); mnr = fmin(mnr, v.x);
    mxi = fmax(mxi, v.y); mni = fmin(mni, v.y);
  }
  __shared__ double s[4][32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mxr = fmax(mxr, __shfl_xor_sync(0xffffffffu, mxr, o));
    mnr = fmin(mnr, __shfl_xor_sync(0xffffffffu, mnr, o));
    mxi = fmax(mxi, __shfl_xor_sync(0xffffffffu, mxi, o));
    mni = fmin(mni, __shfl_xor_sync(0xffffffffu, mni, o));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) { s[0][warp] = mxr; s[1][warp] = mnr; s[2][warp] = mxi; s[3][warp] = mni; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      mxr = fmax(mxr, s[0][w]); mnr = fmin(mnr, s[1][w]);
      mxi = fmax(mxi, s[2][w]); mni = fmin(mni, s[3][w]);
    }
    lam[leaf] = make_double2(0.5 * (mxr + mnr), 0.5 * (mxi + mni));
  }
}

// B^leaf = R~^leaf[internal face rows][external face cols] for the leaves of a batch,
// stored transposed (column-major: column c holds the nint q^2 rows, ld rup4(nint q^2))
// so that stage B reads it with one thread per row, coalesced.
template <class T>
__global__ void extract_b_kernel(const T* Rt, long long rstride, int ldr, const int* leaf_ids,
                                 int nbatch, int q, const uint8_t* int_mask, const long long* b_off,
                                 double2* B64, float2* B32) {
  const int b = blockIdx.y;
  if (b >= nbatch) return;
  const int leaf = leaf_ids[b];
  const int q2 = q * q;
  const unsigned mask = int_mask[leaf];
  const int nint = __popc(mask), next = 6 - nint;
  if (nint == 0) return;
  int ifaces[6], efaces[6];
  int a = 0, e = 0;
  for (int f = 0; f < 6; ++f) {
    if (mask & (1u << f)) ifaces[a++] = f; else efaces[e++] = f;
  }
  const int ldt = (int)rup4(nint * q2);
  const long long off = b_off[leaf];
  const long long total = (long long)nint * q2 * next * q2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / (next * q2)), c = (int)(t % (next * q2));
    const int rf = ifaces[r / q2], cf = efaces[c / q2];
    const T v = Rt[(long long)b * rstride + (long long)(rf * q2 + r % q2) * ldr + cf * q2 + c % q2];
    const long long o = off + (long long)c * ldt + r;  // stored transposed: column c, row r
    if (B64) B64[o] = cvt<double2>(v);
    if (B32) B32[o] = cvt<float2>(v);
  }
}

// [I + D | I] for each cluster of a batch (row-major, ld = ldw); D couples
// internal slot a (leaf alpha, face k) to the slots of beta = nbr(alpha, k)
// through R~^beta's rows on face k^1.
template <class T>
__global__ void assemble_cluster_kernel(T* W, long long wstride, int ldw, int cl0, int nbatch,
                                        const int* cl_slot_begin, const int* slot_lf,
                                        const int* cl_leaf_begin, const int* cl_leaves,
                                        const T* Rt, long long rstride, int ldr, int leafpos0,
                                        GridDims g, int q) {
  const int b = blockIdx.y;
  if (b >= nbatch) return;
  const int c = cl0 + b;
  const int q2 = q * q;
  const int s0 = cl_slot_begin[c], ns = cl_slot_begin[c + 1] - s0;
  const int nint = ns * q2;
  const int lb = cl_leaf_begin[c], le = cl_leaf_begin[c + 1];
  T* Wb = W + (long long)b * wstride;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nint * nint;
       t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t / nint), col = (int)(t % nint);
    const int sa = row / q2, ja = row % q2;
    const int sb = col / q2, jb = col % q2;
    const int lfa = slot_lf[s0 + sa], lfb = slot_lf[s0 + sb];
    const int alpha = lfa / 6, ka = lfa % 6;
    const int beta_b = lfb / 6, kb = lfb % 6;
    T v = czero<T>();
    if (row == col) v.x = 1;
    const int beta = g.neighbor(alpha, ka);
    if (beta == beta_b) {
      int pos = -1;
      for (int l = lb; l < le; ++l)
        if (cl_leaves[l] == beta) pos = l - leafpos0;
      const T r = Rt[(long long)pos * rstride + (long long)((ka ^ 1) * q2 + ja) * ldr + kb * q2 + jb];
      v.x += r.x;
      v.y += r.y;
    }
    Wb[(long long)row * ldw + col] = v;
    T e = czero<T>();
    if (row == col) e.x = 1;
    Wb[(long long)row * ldw + nint + col] = e;
  }
}

template <class T>
__global__ void extract_kc_kernel(const T* W, long long wstride, int ldw, int cl0, int nbatch,
                                  const int* cl_slot_begin, const long long* kc_off, int q, double2* K64,
                                  float2* K32) {
  const int b = blockIdx.y;
  if (b >= nbatch) return;
  const int c = cl0 + b;
  const int q2 = q * q;
  const int nint = (cl_slot_begin[c + 1] - cl_slot_begin[c]) * q2;
  const int ldk = (int)rup4(nint);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nint * nint;
       t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t / nint), col = (int)(t % nint);
    const T v = W[(long long)b * wstride + (long long)row * ldw + nint + col];
    const long long o = kc_off[c] + (long long)row * ldk + col;
    if (K64) K64[o] = cvt<double2>(v);
    if (K32) K32[o] = cvt<float2>(v);
  }
}

// Right-hand-side columns [s; P^{-1} f] of the leaf systems of a batch (leaves
// leaf0..leaf0+nbatch-1), one column per right-hand side at W[:, n + k].
// P^{-1} maps a face's Gauss-point data F (q x q) to the Chebyshev face nodes:
// Qi F Qi^T.
__global__ void recover_rhs_kernel(double2* W, long long wstride, int ld, int leaf0, int nbatch, const double* tab,
                                   TableLayout tl, const double2* s, const double2* f, int nrhs, long long nint,
                                   long long nf) {
  const int q = tl.q, q2 = q * q, n1 = tl.p - 2, ni = n1 * n1 * n1, nb = 6 * q2, n = ni + nb;
  const int b = blockIdx.y;
  if (b >= nbatch) return;
  const int leaf = leaf0 + b;
  const double* Qi = tab + tl.Qi;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * nrhs; t += gridDim.x * blockDim.x) {
    const int r = t % n, k = t / n;
    double2 v = make_double2(0.0, 0.0);
    if (r < ni) {
      if (s) v = s[k * nint + (long long)leaf * ni + r];
    } else {
      const int jb = r - ni, face = jb / q2, a = jb % q2, a1 = a % q, a2 = a / q;
      const double2* F = f + k * nf + (long long)leaf * nb + (long long)face * q2;
      for (int j2 = 0; j2 < q; ++j2) {
        double2 row = make_double2(0.0, 0.0);
        for (int j1 = 0; j1 < q; ++j1) row = cadd(row, cscale(F[j2 * q + j1], Qi[a1 * q + j1]));
        v = cadd(v, cscale(row, Qi[a2 * q + j2]));
      }
    }
    W[(long long)b * wstride + (long long)r * ld + n + k] = v;
  }
}

__global__ void recover_extract_kernel(const double2* W, long long wstride, int ld, int n, int ni, int leaf0,
                                       int nbatch, int nrhs, long long nint, double2* u, long long nfc,
                                       double2* uf) {
  const int b = blockIdx.y;
  if (b >= nbatch) return;
  const int nb = n - ni;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * nrhs; t += gridDim.x * blockDim.x) {
    const int r = t % n, k = t / n;
    const double2 v = W[(long long)b * wstride + (long long)r * ld + n + k];
    if (r < ni) u[k * nint + (long long)(leaf0 + b) * ni + r] = v;
    else if (uf) uf[k * nfc + (long long)(leaf0 + b) * nb + (r - ni)] = v;
  }
}

// FP16 copy of one complex-float row with one FP32 scale: the row is divided by
// s = max(|re|, |im|) over the row before rounding to half precision.
__device__ __forceinline__ void quantize_row(const float2* src, __half2* dst, int ncols, float* scale, int lane) {
  float m = 0.f;
  for (int c = lane; c < ncols; c += 32) m = fmaxf(m, fmaxf(fabsf(src[c].x), fabsf(src[c].y)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float s = (m > 0.f) ? m : 1.f;
  const float inv = 1.f / s;
  for (int c = lane; c < ncols; c += 32) dst[c] = __floats2half2_rn(src[c].x * inv, src[c].y * inv);
  if (lane == 0) *scale = s;
}

// rows of every distinct K block; row gr = block slot * q^2 + j
__global__ void quantize_kc_kernel(const float2* K32, __half2* K16, float* kscale, const int* slot_cluster,
                                   const int* cl_slot_begin, const long long* kc_off, int q2, long long nrows) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long gr = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); gr < nrows; gr += warps) {
    const int slot = (int)(gr / q2);
    const int c = slot_cluster[slot];
    const int s0 = cl_slot_begin[c];
    const int nint = (cl_slot_begin[c + 1] - s0) * q2;
    const long long off = kc_off[c] + (gr - (long long)s0 * q2) * rup4(nint);
    quantize_row(K32 + off, K16 + off, nint, kscale + gr, lane);
  }
}

// K_c rows of one batch straight from the elimination workspace (columns
// [nint, 2 nint) of each cluster's [I + D | I]) into FP16 with row scales.
__global__ void quantize_kc_ws_kernel(const float2* W, long long wstride, int ldw, int cl0, int nbatch,
                                      const int* cl_slot_begin, const long long* kc_off, int q2, __half2* K16,
                                      float* kscale) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.y;
  if (b >= nbatch) return;
  const int c = cl0 + b;
  const int s0 = cl_slot_begin[c];
  const int nint = (cl_slot_begin[c + 1] - s0) * q2;
  const int ldk = (int)rup4(nint);
  for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nint; r += gridDim.x * (blockDim.x >> 5))
    quantize_row(W + (long long)b * wstride + (long long)r * ldw + nint, K16 + kc_off[c] + (long long)r * ldk, nint,
                 kscale + (long long)s0 * q2 + r, lane);
}

// rows of every distinct B block (stored transposed); row index (block*6 + face)*q^2 + j
// for internal faces: divided by its largest |re|, |im| and rounded to FP16.
__global__ void quantize_b_kernel(const float2* B32, __half2* B16, float* bscale, const int* bc_rep,
                                  const uint8_t* int_mask, const long long* b_off, int q2, long long nrows) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long gr = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); gr < nrows; gr += warps) {
    const int leaf = bc_rep[gr / (6 * q2)];
    const int face = (int)((gr / q2) % 6);
    const int j = (int)(gr % q2);
    const unsigned mask = int_mask[leaf];
    if (!(mask & (1u << face))) continue;
    const int nint = __popc(mask);
    const int rb = __popc(mask & ((1u << face) - 1u));
    const int ncols = (6 - nint) * q2, ldr = (int)rup4(nint * q2), row = rb * q2 + j;
    const long long off = b_off[leaf] + row;
    float m = 0.f;
    for (int c = lane; c < ncols; c += 32) {
      const float2 v = B32[off + (long long)c * ldr];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float sc = (m > 0.f) ? m : 1.f;
    const float inv = 1.f / sc;
    for (int c = lane; c < ncols; c += 32) {
      const float2 v = B32[off + (long long)c * ldr];
      B16[off + (long long)c * ldr] = __floats2half2_rn(v.x * inv, v.y * inv);
    }
    if (lane == 0) bscale[gr] = sc;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
int build_precond_fp16(hps_handle* h, cudaStream_t st) {
  const ClusterTables& ct = h->ct;
  const int q2 = h->q * h->q;
  const long long krows = (long long)ct.kc_slot_begin[ct.nkc] * q2;
  const long long brows = (long long)ct.nbc * 6 * q2;
  if (krows > 0 && h->Kc32) {  // lean mode quantized K_c during the build
    quantize_kc_kernel<<<h->nsm * 8, 256, 0, st>>>(h->Kc32, h->Kc16, h->Kc16s, h->dct.kslot_class,
                                                    h->dct.kc_slot_begin, h->dct.kc_off, q2, krows);
    HPS_CUDA_TRY(cudaGetLastError());
  }
  if (brows > 0) {
    quantize_b_kernel<<<h->nsm * 8, 256, 0, st>>>(h->B32, h->B16, h->B16s, h->dct.bc_rep, h->dct.int_mask,
                                                   h->dct.b_off, q2, brows);
    HPS_CUDA_TRY(cudaGetLastError());
  }
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  return HPS_OK;
}

cudaError_t launch_tables(double* tables, const TableLayout& tl, double hx, double hy, double hz,
                          cudaStream_t st) {
  tables_kernel<<<1, 32, 0, st>>>(tables, tl, hx, hy, hz);
  return cudaGetLastError();
}

cudaError_t launch_cdiag(const double2* b, double kappa, long long count, double2* c, cudaStream_t st) {
  cdiag_kernel<<<1024, 256, 0, st>>>(b, kappa, count, c);
  return cudaGetLastError();
}

cudaError_t launch_nodes(const double* tables, const TableLayout& tl, int nx, int ny, int nz,
                         double* xi, double* xf, double* xc, cudaStream_t st) {
  nodes_kernel<<<1024, 256, 0, st>>>(tables, tl, nx, ny, nz, xi, xf, xc);
  return cudaGetLastError();
}

namespace {

constexpr int kGjThreads = 512;

template <class T>
cudaError_t run_gj(T* W, long long wstride, int ld, int n, int ncols, int gj0, int nbatch, int* status,
                   cudaStream_t st) {
  const size_t smem = (size_t)ncols * sizeof(T);
  cudaError_t e = allow_dynamic_smem((const void*)gj_kernel<T, kGjThreads>, smem);
  if (e != cudaSuccess) return e;
  gj_kernel<T, kGjThreads><<<nbatch, kGjThreads, smem, st>>>(W, wstride, ld, n, ncols, gj0, nbatch, status);
  return cudaGetLastError();
}

template <class T>
cudaError_t run_seg_kron(T* M, long long mstride, int ld, int nrows, int ncols, int nbatch,
                         const double* tables, const TableLayout& tl, int trans, int mode, int nsm, cudaStream_t st) {
  const int q2 = tl.q * tl.q;
  const size_t smem = 8 * 2 * q2 * sizeof(T);
  cudaError_t e = allow_dynamic_smem((const void*)seg_kron_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  seg_kron_kernel<T><<<nsm * 8, 256, smem, st>>>(M, mstride, ld, nrows, ncols, nbatch, tables, tl, trans, mode);
  return cudaGetLastError();
}

// Device status word + copy-back helper.
int check_status(int* d_status, cudaStream_t st, const char* what) {
  int hs = 0;
  HPS_CUDA_TRY(cudaMemcpyAsync(&hs, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  if (hs != 0) {
    set_error(std::string(what) + ": zero pivot in the elimination");
    return HPS_EBREAKDOWN;
  }
  return HPS_OK;
}

size_t workspace_budget(const hps_handle* h) {
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  return std::min(workspace_cap(h), fr / 3);
}

}  // namespace

// Cap on the transient setup workspace: 24 GiB, raised up to 96 GiB where that is needed for one
// leaf elimination per SM (large leaves, p >= 14); the remaining HBM budget of the handle when one
// is set (setup also keeps it under a third of the free device memory).
size_t workspace_cap(const hps_handle* h) {
  const size_t per = (size_t)h->n * (size_t)(h->n + h->nb + h->ni) * sizeof(double2);
  size_t cap = std::max((size_t)24 << 30, std::min(per * (size_t)std::max(h->nsm, 1), (size_t)96 << 30));
  if (h->opt.hbm_budget) {
    const size_t rest = h->opt.hbm_budget > h->bytes ? h->opt.hbm_budget - h->bytes : 0;
    cap = std::min(cap, rest);
  }
  return cap;
}

size_t exact_maps_workspace(const hps_handle* h, size_t budget, int* nbatch_out) {
  const long long per = (long long)h->n * (h->n + h->nb + h->ni) * (long long)sizeof(double2);
  int nbatch = (int)std::min<long long>((long long)h->nl, std::max<long long>(1, (long long)(budget / per)));
  nbatch = std::min(nbatch, 4 * h->nsm);
  if (nbatch_out) *nbatch_out = nbatch;
  return (size_t)per * nbatch;
}

size_t precond_workspace(const hps_handle* h, size_t budget, int* cb_out) {
  const ClusterTables& ct = h->ct;
  const int q2 = h->q * h->q;
  int max_int = 0, max_leaves = 0;
  for (int k = 0; k < ct.nkc; ++k) {
    const int c = ct.kc_rep[k];
    max_int = std::max(max_int, (ct.cl_slot_begin[c + 1] - ct.cl_slot_begin[c]) * q2);
    max_leaves = std::max(max_leaves, ct.cl_leaf_begin[c + 1] - ct.cl_leaf_begin[c]);
  }
  const long long wl_stride = (long long)h->n * (h->n + h->nb);
  const int ldw = std::max(2, 2 * max_int);
  const long long wc_stride = (long long)std::max(1, max_int) * ldw;
  const size_t per_cluster =
      ((size_t)wl_stride * max_leaves + (size_t)h->nb * h->ldR * max_leaves + (size_t)wc_stride) * sizeof(double2);
  int cb = (int)std::min<size_t>((size_t)std::max(1, ct.nkc), std::max<size_t>(1, budget / per_cluster));
  cb = std::min(cb, std::max(1, 2 * h->nsm));
  if (cb_out) *cb_out = cb;
  return per_cluster * cb;
}

// Interior values of the leaf solutions u^tau = A^{tau,-1} [s^tau; P^{-1} f^tau]
// (eq. (leaf)), by FP64 elimination of each leaf system with nrhs extra columns.
int recover_interior(hps_handle* h, const double2* s, const double2* f, int nrhs, double2* u, double2* uf,
                     cudaStream_t st) {
  const int n = h->n, ni = h->ni;
  const int ncols = n + nrhs, ld = ncols;
  const long long wstride = (long long)n * ld;
  const size_t per = (size_t)wstride * sizeof(double2);
  int nbatch = (int)std::min<size_t>((size_t)h->nl, std::max<size_t>(1, workspace_budget(h) / per));
  nbatch = std::min(nbatch, 4 * h->nsm);
  double2* W = nullptr;
  int* d_status = nullptr;
  HPS_CUDA_TRY(cudaMalloc(&W, per * nbatch));
  HPS_CUDA_TRY(cudaMalloc(&d_status, sizeof(int)));
  HPS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  int rc = HPS_OK;
  for (int l0 = 0; l0 < h->nl && rc == HPS_OK; l0 += nbatch) {
    const int nbt = std::min(nbatch, h->nl - l0);
    auto body = [&]() -> int {
      HPS_CUDA_TRY(cudaMemsetAsync(W, 0, per * nbt, st));
      dim3 ga((n + 127) / 128, nbt);
      assemble_kernel<double2><<<ga, 128, 0, st>>>(W, wstride, ld, nullptr, l0, nbt, h->tables, h->tl, h->eta,
                                                  h->cdiag, nullptr, 0);
      HPS_CUDA_TRY(cudaGetLastError());
      recover_rhs_kernel<<<dim3(32, nbt), 128, 0, st>>>(W, wstride, ld, l0, nbt, h->tables, h->tl, s, f, nrhs,
                                                         h->nint, h->nf);
      HPS_CUDA_TRY(cudaGetLastError());
      HPS_CUDA_TRY(run_gj(W, wstride, ld, n, ncols, 0, nbt, d_status, st));
      recover_extract_kernel<<<dim3(32, nbt), 128, 0, st>>>(W, wstride, ld, n, ni, l0, nbt, nrhs, h->nint, u,
                                                             (long long)h->nl * h->nb, uf);
      HPS_CUDA_TRY(cudaGetLastError());
      return HPS_OK;
    };
    rc = body();
  }
  if (rc == HPS_OK) rc = check_status(d_status, st, "leaf solution recovery");
  cudaStreamSynchronize(st);
  cudaFree(W);
  cudaFree(d_status);
  return rc;
}

int build_exact_maps(hps_handle* h, const double2* cdiag, cudaStream_t st) {
  const int n = h->n, ni = h->ni, nb = h->nb;
  const int ncols = n + nb + ni;
  const int ld = ncols;
  const long long wstride = (long long)n * ld;
  const size_t per = (size_t)wstride * sizeof(double2);
  int nbatch = 1;
  exact_maps_workspace(h, workspace_budget(h), &nbatch);
  double2* W = nullptr;
  int* d_status = nullptr;
  double2 *Rtmp = nullptr, *Htmp = nullptr;  // lean mode: FP64 maps of one batch before rounding
  HPS_CUDA_TRY(cudaMalloc(&W, per * nbatch));
  HPS_CUDA_TRY(cudaMalloc(&d_status, sizeof(int)));
  HPS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  if (!h->R64) {
    HPS_CUDA_TRY(cudaMalloc(&Rtmp, (size_t)nbatch * nb * h->ldR * sizeof(double2)));
    HPS_CUDA_TRY(cudaMalloc(&Htmp, (size_t)nbatch * nb * h->ldH * sizeof(double2)));
    HPS_CUDA_TRY(cudaMemsetAsync(Rtmp, 0, (size_t)nbatch * nb * h->ldR * sizeof(double2), st));
    HPS_CUDA_TRY(cudaMemsetAsync(Htmp, 0, (size_t)nbatch * nb * h->ldH * sizeof(double2), st));
  }
  int rc = HPS_OK;
  for (int l0 = 0; l0 < h->nl && rc == HPS_OK; l0 += nbatch) {
    const int nbt = std::min(nbatch, h->nl - l0);
    auto body = [&]() -> int {
      HPS_CUDA_TRY(cudaMemsetAsync(W, 0, per * nbt, st));
      dim3 ga((n + 127) / 128, nbt);
      assemble_kernel<double2><<<ga, 128, 0, st>>>(W, wstride, ld, nullptr, l0, nbt, h->tables, h->tl, h->eta,
                                                  cdiag, nullptr, 2);
      HPS_CUDA_TRY(cudaGetLastError());
      HPS_CUDA_TRY(run_gj(W, wstride, ld, n, ncols, ni, nbt, d_status, st));
      double2* Rb = h->R64 ? h->R64 + (long long)l0 * nb * h->ldR : Rtmp;
      double2* Hb = h->H64 ? h->H64 + (long long)l0 * nb * h->ldH : Htmp;
      dim3 ge(256, nbt);
      extract_kernel<double2><<<ge, 256, 0, st>>>(W, wstride, ld, n, ni, nb, h->eta, nbt, Rb,
                                                  (long long)nb * h->ldR, h->ldR, Hb, (long long)nb * h->ldH, h->ldH);
      HPS_CUDA_TRY(cudaGetLastError());
      // R = P (R_C P^{-1}): rows by Q^{-T} (.) Q^{-1}, then columns by Q (.) Q^T.
      HPS_CUDA_TRY(run_seg_kron(Rb, (long long)nb * h->ldR, h->ldR, nb, nb, nbt, h->tables, h->tl, 1, 0, h->nsm, st));
      HPS_CUDA_TRY(run_seg_kron(Rb, (long long)nb * h->ldR, h->ldR, nb, nb, nbt, h->tables, h->tl, 0, 1, h->nsm, st));
      HPS_CUDA_TRY(run_seg_kron(Hb, (long long)nb * h->ldH, h->ldH, nb, ni, nbt, h->tables, h->tl, 0, 1, h->nsm, st));
      if (h->R32) {
        const long long cnt = (long long)nbt * nb * h->ldR;
        cast_kernel<<<1024, 256, 0, st>>>(Rb, h->R32 + (long long)l0 * nb * h->ldR, cnt);
        HPS_CUDA_TRY(cudaGetLastError());
      }
      if (h->H32) {
        const long long cnt = (long long)nbt * nb * h->ldH;
        cast_kernel<<<1024, 256, 0, st>>>(Hb, h->H32 + (long long)l0 * nb * h->ldH, cnt);
        HPS_CUDA_TRY(cudaGetLastError());
      }
      // lean mode: the FP16 remainders that make the FP32 maps FP64-accurate
      if (h->R16lo)
        HPS_CUDA_TRY(launch_split_lo(Rb, (long long)nbt * nb, h->ldR, h->R16lo + (long long)l0 * nb * h->ldR,
                                     h->R16ls + (long long)l0 * nb, st));
      if (h->H16lo)
        HPS_CUDA_TRY(launch_split_lo(Hb, (long long)nbt * nb, h->ldH, h->H16lo + (long long)l0 * nb * h->ldH,
                                     h->H16ls + (long long)l0 * nb, st));
      return HPS_OK;
    };
    rc = body();
  }
  if (rc == HPS_OK) rc = check_status(d_status, st, "leaf ItI maps");
  cudaStreamSynchronize(st);
  cudaFree(W);
  cudaFree(d_status);
  if (Rtmp) cudaFree(Rtmp);
  if (Htmp) cudaFree(Htmp);
  return rc;
}

void build_cluster_tables(hps_handle* h, int width) {
  ClusterTables& ct = h->ct;
  ct = ClusterTables();
  ct.lf_slot.assign((size_t)h->nl * 6, -1);
  ct.int_mask.assign(h->nl, 0);
  ct.b_off.assign(h->nl, 0);
  ct.cl_leaf_begin.push_back(0);
  ct.cl_slot_begin.push_back(0);
  auto lid = [&](int ix, int iy, int iz) { return ix + h->nx * (iy + h->ny * iz); };
  for (int cz = 0; cz < h->nz; cz += width)
    for (int cy = 0; cy < h->ny; cy += width)
      for (int cx = 0; cx < h->nx; cx += width) {
        const int c = ct.ncl++;
        const int x1 = std::min(cx + width, h->nx), y1 = std::min(cy + width, h->ny), z1 = std::min(cz + width, h->nz);
        for (int iz = cz; iz < z1; ++iz)
          for (int iy = cy; iy < y1; ++iy)
            for (int ix = cx; ix < x1; ++ix) ct.cl_leaves.push_back(lid(ix, iy, iz));
        for (int iz = cz; iz < z1; ++iz)
          for (int iy = cy; iy < y1; ++iy)
            for (int ix = cx; ix < x1; ++ix) {
              const int leaf = lid(ix, iy, iz);
              const int c3[3] = {ix, iy, iz}, lo3[3] = {cx, cy, cz}, hi3[3] = {x1, y1, z1};
              for (int f = 0; f < 6; ++f) {
                const int axis = f >> 1, d = (f & 1) ? 1 : -1;
                const int v = c3[axis] + d;
                if (v < lo3[axis] || v >= hi3[axis]) continue;
                const int slot = ct.nslots++;
                ct.slot_lf.push_back(leaf * 6 + f);
                ct.slot_cluster.push_back(c);
                ct.lf_slot[(size_t)leaf * 6 + f] = slot;
                ct.int_mask[leaf] |= (uint8_t)(1u << f);
              }
            }
        ct.cl_leaf_begin.push_back((int)ct.cl_leaves.size());
        ct.cl_slot_begin.push_back(ct.nslots);
      }
  ct.max_ext = 0;
  for (int leaf = 0; leaf < h->nl; ++leaf) ct.max_ext = std::max(ct.max_ext, 6 - __builtin_popcount(ct.int_mask[leaf]));
  ct.leaf_cluster.assign(h->nl, 0);
  for (int c = 0; c < ct.ncl; ++c)
    for (int l = ct.cl_leaf_begin[c]; l < ct.cl_leaf_begin[c + 1]; ++l) ct.leaf_cluster[ct.cl_leaves[l]] = c;
  assign_blocks(h, nullptr);
}

// Distinct preconditioner blocks.  With lamq == nullptr every cluster and leaf
// owns its block (the sizes hps_setup_bytes reserves); otherwise leaves are
// keyed by (binned lambda, internal-face mask) and clusters by the sequence of
// their leaves' keys, which fixes the cluster's shape and its J_c exactly.
void assign_blocks(hps_handle* h, const std::vector<double2>* lamq) {
  ClusterTables& ct = h->ct;
  const int q2 = h->q * h->q;
  auto bits = [](double v) {
    v += 0.0;  // -0 and +0 are one constant
    uint64_t u;
    std::memcpy(&u, &v, sizeof(u));
    return u;
  };
  // B blocks
  ct.leaf_bcls.assign(h->nl, 0);
  ct.bc_rep.clear();
  std::map<std::tuple<uint64_t, uint64_t, int>, int> bkeys;
  for (int leaf = 0; leaf < h->nl; ++leaf) {
    int cls;
    if (!lamq) {
      cls = (int)ct.bc_rep.size();
      ct.bc_rep.push_back(leaf);
    } else {
      const double2 l = (*lamq)[leaf];
      auto key = std::make_tuple(bits(l.x), bits(l.y), (int)ct.int_mask[leaf]);
      auto it = bkeys.find(key);
      if (it == bkeys.end()) {
        cls = (int)ct.bc_rep.size();
        bkeys.emplace(key, cls);
        ct.bc_rep.push_back(leaf);
      } else {
        cls = it->second;
      }
    }
    ct.leaf_bcls[leaf] = cls;
  }
  ct.nbc = (int)ct.bc_rep.size();
  std::vector<long long> bc_off(ct.nbc);
  long long off = 0;
  for (int k = 0; k < ct.nbc; ++k) {
    const int ni_ = __builtin_popcount(ct.int_mask[ct.bc_rep[k]]);
    bc_off[k] = off;
    off += (long long)(6 - ni_) * q2 * round_up((long long)ni_ * q2, 4);
  }
  ct.b_elems = off;
  ct.b_off.assign(h->nl, 0);
  for (int leaf = 0; leaf < h->nl; ++leaf) ct.b_off[leaf] = bc_off[ct.leaf_bcls[leaf]];
  // K blocks
  ct.cl_class.assign(ct.ncl, 0);
  ct.kc_rep.clear();
  std::map<std::vector<uint64_t>, int> kkeys;
  for (int c = 0; c < ct.ncl; ++c) {
    int cls;
    if (!lamq) {
      cls = (int)ct.kc_rep.size();
      ct.kc_rep.push_back(c);
    } else {
      std::vector<uint64_t> key;
      for (int l = ct.cl_leaf_begin[c]; l < ct.cl_leaf_begin[c + 1]; ++l) {
        const int leaf = ct.cl_leaves[l];
        const double2 v = (*lamq)[leaf];
        key.push_back(bits(v.x));
        key.push_back(bits(v.y));
        key.push_back(ct.int_mask[leaf]);
      }
      auto it = kkeys.find(key);
      if (it == kkeys.end()) {
        cls = (int)ct.kc_rep.size();
        kkeys.emplace(std::move(key), cls);
        ct.kc_rep.push_back(c);
      } else {
        cls = it->second;
      }
    }
    ct.cl_class[c] = cls;
  }
  ct.nkc = (int)ct.kc_rep.size();
  ct.kc_slot_begin.assign(ct.nkc + 1, 0);
  ct.kc_off.assign(ct.nkc, 0);
  off = 0;
  for (int k = 0; k < ct.nkc; ++k) {
    const int c = ct.kc_rep[k];
    const int ns = ct.cl_slot_begin[c + 1] - ct.cl_slot_begin[c];
    const long long nint = (long long)ns * q2;
    ct.kc_slot_begin[k + 1] = ct.kc_slot_begin[k] + ns;
    ct.kc_off[k] = off;
    off += nint * round_up(nint, 4);
  }
  ct.kc_elems = off;
  ct.cl_kc_off.assign(ct.ncl, 0);
  for (int c = 0; c < ct.ncl; ++c) ct.cl_kc_off[c] = ct.kc_off[ct.cl_class[c]];
  ct.kslot_class.assign(ct.kc_slot_begin[ct.nkc], 0);
  for (int k = 0; k < ct.nkc; ++k)
    for (int s = ct.kc_slot_begin[k]; s < ct.kc_slot_begin[k + 1]; ++s) ct.kslot_class[s] = k;
  // members of each block and the stage-K work items
  ct.kc_mem_begin.assign(ct.nkc + 1, 0);
  for (int c = 0; c < ct.ncl; ++c) ++ct.kc_mem_begin[ct.cl_class[c] + 1];
  for (int k = 0; k < ct.nkc; ++k) ct.kc_mem_begin[k + 1] += ct.kc_mem_begin[k];
  ct.kc_members.assign(ct.ncl, 0);
  {
    std::vector<int> fill(ct.kc_mem_begin.begin(), ct.kc_mem_begin.end() - 1);
    for (int c = 0; c < ct.ncl; ++c) ct.kc_members[fill[ct.cl_class[c]]++] = c;
  }
  // widest member group whose staged vectors (complex double in the FP64 form)
  // fit in shared memory: W * (xcap + q^2) * 16 bytes
  int xcap = std::max(h->nb, h->ni);
  for (int c = 0; c < ct.ncl; ++c) xcap = std::max(xcap, (ct.cl_slot_begin[c + 1] - ct.cl_slot_begin[c]) * q2);
  xcap = (int)round_up(xcap, 64);
  int wmax = 8;
  while (wmax > 1 && (size_t)wmax * (xcap + q2) * 16 > (size_t)220 * 1024) wmax >>= 1;
  // class-ordered stage-K input layout
  ct.cl_tpos.assign(ct.ncl, 0);
  ct.lf_tpos.assign((size_t)h->nl * 6, -1);
  {
    long long pos = 0;
    for (int k = 0; k < ct.nkc; ++k) {
      pos = round_up(pos, 16);
      for (int m = ct.kc_mem_begin[k]; m < ct.kc_mem_begin[k + 1]; ++m) {
        const int c = ct.kc_members[m];
        ct.cl_tpos[c] = pos;
        for (int sl = ct.cl_slot_begin[c]; sl < ct.cl_slot_begin[c + 1]; ++sl)
          ct.lf_tpos[ct.slot_lf[sl]] = pos + (long long)(sl - ct.cl_slot_begin[c]) * q2;
        pos += (long long)(ct.cl_slot_begin[c + 1] - ct.cl_slot_begin[c]) * q2;
      }
    }
    ct.tsize = round_up(std::max<long long>(pos, 1), 16);
  }
  // stage-B offsets
  ct.brd.assign((size_t)h->nl * 6, 0);
  ct.bto.assign((size_t)h->nl * 6, 0);
  ct.bsc.assign((size_t)h->nl * 6, 0);
  for (int leaf = 0; leaf < h->nl; ++leaf) {
    const int ix = leaf % h->nx, iy = (leaf / h->nx) % h->ny, iz = leaf / (h->nx * h->ny);
    int k = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int f = 0; f < 6; ++f) {
        const bool internal = (ct.int_mask[leaf] >> f) & 1;
        if (internal != (pass == 0)) continue;
        const size_t e = (size_t)leaf * 6 + k++;
        if (internal) {
          int c3[3] = {ix, iy, iz};
          c3[f >> 1] += (f & 1) ? 1 : -1;
          const int nbr = c3[0] + h->nx * (c3[1] + h->ny * c3[2]);
          ct.brd[e] = nbr * h->nb + (f ^ 1) * q2;
          ct.bto[e] = (int)ct.lf_tpos[(size_t)nbr * 6 + (f ^ 1)];
          ct.bsc[e] = (ct.leaf_bcls[leaf] * 6 + f) * q2;
        } else {
          ct.brd[e] = leaf * h->nb + f * q2;
        }
      }
  }
  // stage-B groups: leaves of one B block (ascending), kBGroup at a time; with one leaf per
  // group, in leaf order (neighbouring leaves on neighbouring CTAs write neighbouring t slots)
  {
    std::vector<std::vector<int>> by_class(kBGroup > 1 ? ct.nbc : 1);
    for (int leaf = 0; leaf < h->nl; ++leaf) by_class[kBGroup > 1 ? ct.leaf_bcls[leaf] : 0].push_back(leaf);
    ct.bgroup_leaves.clear();
    ct.bgroups.clear();
    ct.max_group = 0;
    for (const auto& ls : by_class)
      for (size_t i = 0; i < ls.size(); i += kBGroup) {
        const int cnt = (int)std::min<size_t>(kBGroup, ls.size() - i);
        ct.bgroups.push_back(make_int2((int)ct.bgroup_leaves.size(), cnt));
        ct.max_group = std::max(ct.max_group, cnt);
        for (int g = 0; g < cnt; ++g) ct.bgroup_leaves.push_back(ls[i + g]);
      }
  }
  // one 3D array of blocks and one [position][nint] matrix of t (multi-RHS stage K)
  ct.pos_class.assign(ct.ncl, 0);
  for (int m = 0; m < ct.ncl; ++m) ct.pos_class[m] = ct.cl_class[ct.kc_members[m]];
  ct.uniform = ct.nkc > 0;
  {
    const long long nint0 = ct.nkc > 0 ? (long long)(ct.kc_slot_begin[1] - ct.kc_slot_begin[0]) * q2 : 0;
    if (nint0 == 0 || nint0 % 16 != 0) ct.uniform = false;
    for (int k = 0; k < ct.nkc && ct.uniform; ++k)
      if ((long long)(ct.kc_slot_begin[k + 1] - ct.kc_slot_begin[k]) * q2 != nint0 || ct.kc_off[k] != (long long)k * nint0 * nint0)
        ct.uniform = false;
    for (int m = 0; m < ct.ncl && ct.uniform; ++m)
      if (ct.cl_tpos[ct.kc_members[m]] != m * nint0) ct.uniform = false;
    ct.nint0 = ct.uniform ? (int)nint0 : 0;
  }
  // FP16 tensor-core stage K items of one right-hand side: per block, per 128-row tile, the
  // members in tiles of 64 (consecutive items reuse the block's row tile from L2)
  ct.tc16_items.clear();
  if (ct.uniform && ct.nint0 % 32 == 0) {
    const int mtiles = (ct.nint0 + 127) / 128;
    for (int k = 0; k < ct.nkc; ++k)
      for (int mt = 0; mt < mtiles; ++mt)
        for (int p0 = ct.kc_mem_begin[k]; p0 < ct.kc_mem_begin[k + 1]; p0 += 64)
          ct.tc16_items.push_back(make_int4(k, mt, p0, std::min(64, ct.kc_mem_begin[k + 1] - p0)));
  }
  // blocks for the tensor-core path: many members, an even row length (16-byte
  // aligned member rows of complex floats)
  ct.kc_tc.clear();
  for (int k = 0; k < ct.nkc; ++k) {
    const int ns = ct.kc_slot_begin[k + 1] - ct.kc_slot_begin[k];
    const int nmem = ct.kc_mem_begin[k + 1] - ct.kc_mem_begin[k];
    if (lamq && ns > 0 && nmem >= kTcMinMembers && ((long long)ns * q2) % 2 == 0) ct.kc_tc.push_back(k);
  }
  // items of the tensor-core blocks go last in every bucket, so that the first
  // kitems_ntc[g] items are the rest
  for (auto& v : ct.kitems) v.clear();
  std::vector<char> is_tc(ct.nkc, 0);
  for (int k : ct.kc_tc) is_tc[k] = 1;
  for (int pass = 0; pass < 2; ++pass) {
    for (int k = 0; k < ct.nkc; ++k) {
      const int ns = ct.kc_slot_begin[k + 1] - ct.kc_slot_begin[k];
      if (ns == 0 || is_tc[k] != pass) continue;
      int pos = ct.kc_mem_begin[k];
      const int end = ct.kc_mem_begin[k + 1];
      while (pos < end) {
        const int cnt = std::min(end - pos, wmax);
        int bucket = 0;
        while ((1 << bucket) < cnt) ++bucket;
        for (int sl = 0; sl < ns; ++sl)
          for (int part = 0; part < kKRowSplit; ++part)
            ct.kitems[bucket].push_back(make_int4(k, sl * kKRowSplit + part, pos, cnt));
        pos += cnt;
      }
    }
    if (pass == 0)
      for (int g = 0; g < 4; ++g) ct.kitems_ntc[g] = (long long)ct.kitems[g].size();
  }
}

// The distinct cluster blocks, built with elimination in T: complex double
// when the FP64 form is kept, complex float otherwise (the FP32 elimination
// gives the boundary block of the inverse to ~2e-7, far below what a
// preconditioner needs, at the FP32 rate).  One representative cluster per
// block is built; its leaves' B blocks are the distinct B blocks (a leaf's B
// block depends only on its binned lambda and internal-face mask, both part of
// the cluster key).  rep_* index the representatives as clusters 0..nkc-1.
template <class T>
int build_precond_blocks(hps_handle* h, const int* d_rep_leaf_begin, const int* d_rep_leaves,
                         const int* d_rep_slot_lf, const std::vector<int>& rep_leaf_begin, cudaStream_t st) {
  ClusterTables& ct = h->ct;
  const int n = h->n, ni = h->ni, nb = h->nb, q = h->q, q2 = q * q;
  int max_int = 0, max_leaves = 0;
  for (int k = 0; k < ct.nkc; ++k) {
    max_int = std::max(max_int, (ct.kc_slot_begin[k + 1] - ct.kc_slot_begin[k]) * q2);
    max_leaves = std::max(max_leaves, rep_leaf_begin[k + 1] - rep_leaf_begin[k]);
  }
  const int ncols_l = n + nb, ld_l = ncols_l;
  const long long wl_stride = (long long)n * ld_l;
  const int ldw = std::max(2, 2 * max_int);
  const long long wc_stride = (long long)std::max(1, max_int) * ldw;
  int cb = 1;
  precond_workspace(h, workspace_budget(h), &cb);
  T *Wl = nullptr, *Rt = nullptr, *Wc = nullptr;
  int* d_status = nullptr;
  HPS_CUDA_TRY(cudaMalloc(&Wl, (size_t)wl_stride * max_leaves * cb * sizeof(T)));
  HPS_CUDA_TRY(cudaMalloc(&Rt, (size_t)nb * h->ldR * max_leaves * cb * sizeof(T)));
  HPS_CUDA_TRY(cudaMalloc(&Wc, (size_t)wc_stride * cb * sizeof(T)));
  HPS_CUDA_TRY(cudaMalloc(&d_status, sizeof(int)));
  HPS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  GridDims gd{h->nx, h->ny, h->nz};
  int rc = HPS_OK;
  for (int c0 = 0; c0 < ct.nkc && rc == HPS_OK; c0 += cb) {
    const int nc = std::min(cb, ct.nkc - c0);
    const int lb = rep_leaf_begin[c0], le = rep_leaf_begin[c0 + nc];
    const int nlb = le - lb;
    const int* leaf_ids = d_rep_leaves + lb;
    auto body = [&]() -> int {
      HPS_CUDA_TRY(cudaMemsetAsync(Wl, 0, (size_t)wl_stride * nlb * sizeof(T), st));
      dim3 ga((n + 127) / 128, nlb);
      assemble_kernel<T><<<ga, 128, 0, st>>>(Wl, wl_stride, ld_l, leaf_ids, 0, nlb, h->tables, h->tl, h->eta,
                                             nullptr, h->lambda_q, 1);
      HPS_CUDA_TRY(cudaGetLastError());
      HPS_CUDA_TRY(run_gj(Wl, wl_stride, ld_l, n, ncols_l, ni, nlb, d_status, st));
      dim3 ge(256, nlb);
      extract_kernel<T><<<ge, 256, 0, st>>>(Wl, wl_stride, ld_l, n, ni, nb, h->eta, nlb, Rt, (long long)nb * h->ldR,
                                            h->ldR, nullptr, 0, 0);
      HPS_CUDA_TRY(cudaGetLastError());
      HPS_CUDA_TRY(run_seg_kron(Rt, (long long)nb * h->ldR, h->ldR, nb, nb, nlb, h->tables, h->tl, 1, 0, h->nsm, st));
      HPS_CUDA_TRY(run_seg_kron(Rt, (long long)nb * h->ldR, h->ldR, nb, nb, nlb, h->tables, h->tl, 0, 1, h->nsm, st));
      extract_b_kernel<T><<<dim3(64, nlb), 256, 0, st>>>(Rt, (long long)nb * h->ldR, h->ldR, leaf_ids, nlb, q,
                                                         h->dct.int_mask, h->dct.b_off, h->B64, h->B32);
      HPS_CUDA_TRY(cudaGetLastError());
      assemble_cluster_kernel<T><<<dim3(256, nc), 256, 0, st>>>(Wc, wc_stride, ldw, c0, nc, h->dct.kc_slot_begin,
                                                                d_rep_slot_lf, d_rep_leaf_begin, d_rep_leaves, Rt,
                                                                (long long)nb * h->ldR, h->ldR, lb, gd, q);
      HPS_CUDA_TRY(cudaGetLastError());
      // blocks of one size are eliminated in one launch
      int cstart = c0;
      while (cstart < c0 + nc) {
        const int sz = (ct.kc_slot_begin[cstart + 1] - ct.kc_slot_begin[cstart]) * q2;
        int cend = cstart + 1;
        while (cend < c0 + nc && (ct.kc_slot_begin[cend + 1] - ct.kc_slot_begin[cend]) * q2 == sz) ++cend;
        if (sz > 0)
          HPS_CUDA_TRY(run_gj(Wc + (long long)(cstart - c0) * wc_stride, wc_stride, ldw, sz, 2 * sz, 0, cend - cstart,
                              d_status, st));
        cstart = cend;
      }
      if (h->Kc64 || h->Kc32) {
        extract_kc_kernel<T><<<dim3(256, nc), 256, 0, st>>>(Wc, wc_stride, ldw, c0, nc, h->dct.kc_slot_begin,
                                                            h->dct.kc_off, q, h->Kc64, h->Kc32);
        HPS_CUDA_TRY(cudaGetLastError());
      }
      if constexpr (std::is_same<T, float2>::value) {
        if (!h->Kc32 && h->Kc16) {
          quantize_kc_ws_kernel<<<dim3(64, nc), 256, 0, st>>>(Wc, wc_stride, ldw, c0, nc, h->dct.kc_slot_begin,
                                                              h->dct.kc_off, q2, h->Kc16, h->Kc16s);
          HPS_CUDA_TRY(cudaGetLastError());
        }
      }
      return HPS_OK;
    };
    rc = body();
  }
  if (rc == HPS_OK) rc = check_status(d_status, st, "preconditioner blocks");
  cudaStreamSynchronize(st);
  cudaFree(Wl);
  cudaFree(Rt);
  cudaFree(Wc);
  cudaFree(d_status);
  return rc;
}

namespace {
template <class V>
int upload(hps_handle* h, V*& dst, const std::vector<V>& vec, cudaStream_t st) {
  const size_t bytes = std::max<size_t>(1, vec.size()) * sizeof(V);
  HPS_CUDA_TRY(cudaMalloc((void**)&dst, bytes));
  h->bytes += bytes;
  if (!vec.empty()) HPS_CUDA_TRY(cudaMemcpyAsync((void*)dst, vec.data(), vec.size() * sizeof(V), cudaMemcpyHostToDevice, st));
  return HPS_OK;
}
}  // namespace

// lambda^tau of every leaf (h->lambda) and its binned value (h->lambda_q); the
// binned values are returned on the host.  Computed once per handle.
int compute_lambdas(hps_handle* h, const double2* cdiag, cudaStream_t st, std::vector<double2>& lamq) {
  lamq.assign(h->nl, make_double2(0.0, 0.0));
  if (h->lambda_q) {
    HPS_CUDA_TRY(cudaMemcpyAsync(lamq.data(), h->lambda_q, (size_t)h->nl * sizeof(double2), cudaMemcpyDeviceToHost,
                                 st));
    HPS_CUDA_TRY(cudaStreamSynchronize(st));
    return HPS_OK;
  }
  HPS_CUDA_TRY(cudaMalloc(&h->lambda_q, (size_t)h->nl * sizeof(double2)));
  h->bytes += (size_t)h->nl * sizeof(double2);
  lambda_kernel<<<h->nl, 256, 0, st>>>(cdiag, h->ni, h->lambda);
  HPS_CUDA_TRY(cudaGetLastError());
  std::vector<double2> lam(h->nl);
  HPS_CUDA_TRY(cudaMemcpyAsync(lam.data(), h->lambda, (size_t)h->nl * sizeof(double2), cudaMemcpyDeviceToHost, st));
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  // binning: nearest multiple of w = lambda_bin * max |lambda| (ties to even)
  double w = 0.0;
  if (h->opt.lambda_bin > 0.0) {
    double mx = 0.0;
    for (const double2& l : lam) mx = std::max(mx, std::hypot(l.x, l.y));
    w = h->opt.lambda_bin * mx;
  }
  lamq = lam;
  if (w > 0.0)
    for (double2& l : lamq) l = make_double2(w * std::nearbyint(l.x / w), w * std::nearbyint(l.y / w));
  HPS_CUDA_TRY(cudaMemcpyAsync(h->lambda_q, lamq.data(), (size_t)h->nl * sizeof(double2), cudaMemcpyHostToDevice, st));
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  return HPS_OK;
}

int classify_preconditioner(hps_handle* h, const double2* cdiag, cudaStream_t st) {
  ClusterTables& ct = h->ct;
  int rc;
  std::vector<double2> lamq;
  if ((rc = compute_lambdas(h, cdiag, st, lamq))) return rc;
  assign_blocks(h, &lamq);
  if ((rc = upload(h, h->dct.slot_lf, ct.slot_lf, st))) return rc;
  if ((rc = upload(h, h->dct.slot_cluster, ct.slot_cluster, st))) return rc;
  if ((rc = upload(h, h->dct.cl_slot_begin, ct.cl_slot_begin, st))) return rc;
  if ((rc = upload(h, h->dct.cl_kc_off, ct.cl_kc_off, st))) return rc;
  if ((rc = upload(h, h->dct.lf_slot, ct.lf_slot, st))) return rc;
  if ((rc = upload(h, h->dct.int_mask, ct.int_mask, st))) return rc;
  if ((rc = upload(h, h->dct.b_off, ct.b_off, st))) return rc;
  if ((rc = upload(h, h->dct.leaf_bcls, ct.leaf_bcls, st))) return rc;
  if ((rc = upload(h, h->dct.bc_rep, ct.bc_rep, st))) return rc;
  if ((rc = upload(h, h->dct.kc_off, ct.kc_off, st))) return rc;
  if ((rc = upload(h, h->dct.kc_slot_begin, ct.kc_slot_begin, st))) return rc;
  if ((rc = upload(h, h->dct.kslot_class, ct.kslot_class, st))) return rc;
  if ((rc = upload(h, h->dct.kc_members, ct.kc_members, st))) return rc;
  if ((rc = upload(h, h->dct.cl_tpos, ct.cl_tpos, st))) return rc;
  if ((rc = upload(h, h->dct.lf_tpos, ct.lf_tpos, st))) return rc;
  if ((rc = upload(h, h->dct.brd, ct.brd, st))) return rc;
  if ((rc = upload(h, h->dct.bto, ct.bto, st))) return rc;
  if ((rc = upload(h, h->dct.bsc, ct.bsc, st))) return rc;
  if ((rc = upload(h, h->dct.pos_class, ct.pos_class, st))) return rc;
  if ((rc = upload(h, h->dct.leaf_cluster, ct.leaf_cluster, st))) return rc;
  if ((rc = upload(h, h->dct.tc16_items, ct.tc16_items, st))) return rc;
  if ((rc = upload(h, h->dct.bgroup_leaves, ct.bgroup_leaves, st))) return rc;
  if ((rc = upload(h, h->dct.bgroups, ct.bgroups, st))) return rc;
  for (int i = 0; i < 4; ++i)
    if ((rc = upload(h, h->dct.kitems[i], ct.kitems[i], st))) return rc;
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  return HPS_OK;
}

int build_preconditioner(hps_handle* h, const double2* cdiag, cudaStream_t st) {
  (void)cdiag;
  const ClusterTables& ct = h->ct;
  // the representative cluster of every distinct K block, as clusters 0..nkc-1
  std::vector<int> rep_leaf_begin(1, 0), rep_leaves, rep_slot_lf;
  for (int k = 0; k < ct.nkc; ++k) {
    const int c = ct.kc_rep[k];
    for (int l = ct.cl_leaf_begin[c]; l < ct.cl_leaf_begin[c + 1]; ++l) rep_leaves.push_back(ct.cl_leaves[l]);
    rep_leaf_begin.push_back((int)rep_leaves.size());
    for (int sl = ct.cl_slot_begin[c]; sl < ct.cl_slot_begin[c + 1]; ++sl) rep_slot_lf.push_back(ct.slot_lf[sl]);
  }
  int *d_leaf_begin = nullptr, *d_leaves = nullptr, *d_slot_lf = nullptr;
  auto dev = [&](int*& d, const std::vector<int>& v) -> int {
    HPS_CUDA_TRY(cudaMalloc(&d, std::max<size_t>(1, v.size()) * sizeof(int)));
    if (!v.empty()) HPS_CUDA_TRY(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    return HPS_OK;
  };
  int rc = dev(d_leaf_begin, rep_leaf_begin);
  if (!rc) rc = dev(d_leaves, rep_leaves);
  if (!rc) rc = dev(d_slot_lf, rep_slot_lf);
  if (!rc)
    rc = h->Kc64 ? build_precond_blocks<double2>(h, d_leaf_begin, d_leaves, d_slot_lf, rep_leaf_begin, st)
                 : build_precond_blocks<float2>(h, d_leaf_begin, d_leaves, d_slot_lf, rep_leaf_begin, st);
  cudaStreamSynchronize(st);
  if (d_leaf_begin) cudaFree(d_leaf_begin);
  if (d_leaves) cudaFree(d_leaves);
  if (d_slot_lf) cudaFree(d_slot_lf);
  return rc;
}

// ---------------------------------------------------------------------------
// The paper's own iterative path on the global system (Sec. 3-4): per distinct
// homogenized constant, S~^{-1} = (A~^{-1})_bb (the inverse of the Schur
// complement F_bb - F_bi A~_ii^{-1} A_ib of eq. (block_pc) is the boundary
// block of the inverse of the homogenized leaf matrix), and per axis the
// eigen-decomposition L1 = V E V^{-1} of Algorithm 3.
// ---------------------------------------------------------------------------
namespace {

__global__ void extract_sinv_kernel(const double2* W, long long wstride, int ld, int n, int ni, int nb, int nbatch,
                                    const int* cls, double2* S64, float2* S32) {
  const int b = blockIdx.y;
  if (b >= nbatch) return;
  const long long off = (long long)cls[b] * nb * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nb * nb;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / nb), c = (int)(t % nb);
    const double2 v = W[(long long)b * wstride + (long long)(ni + r) * ld + n + c];
    if (S64) S64[off + t] = v;
    if (S32) S32[off + t] = make_float2((float)v.x, (float)v.y);
  }
}

// Real eigen-decomposition M = V diag(E) V^{-1} of a small matrix with real,
// distinct eigenvalues (the interior block of the squared Chebyshev
// differentiation matrix): QR iteration with the last diagonal entry as shift
// and deflation, then inverse iteration for each eigenvector and Gauss-Jordan
// for V^{-1}.  Returns false when it does not converge or does not reproduce M.
bool small_eig(int n, const std::vector<double>& M, std::vector<double>& V, std::vector<double>& Vi,
               std::vector<double>& E) {
  auto at = [n](std::vector<double>& A, int i, int j) -> double& { return A[(size_t)i * n + j]; };
  std::vector<double> T(M);
  double nrm = 0.0;
  for (double v : M) nrm = std::max(nrm, std::fabs(v));
  if (nrm == 0.0) return false;
  E.assign(n, 0.0);
  int m = n;
  struct Rot {
    double c, s;
    int i0, i1;
  };
  for (int iter = 0; m > 0 && iter < 100000; ++iter) {
    if (m == 1) {
      E[0] = at(T, 0, 0);
      m = 0;
      break;
    }
    double last = 0.0;
    for (int j = 0; j + 1 < m; ++j) last = std::max(last, std::fabs(at(T, m - 1, j)));
    if (last <= 1e-15 * nrm) {
      E[m - 1] = at(T, m - 1, m - 1);
      --m;
      continue;
    }
    const double mu = at(T, m - 1, m - 1);
    for (int i = 0; i < m; ++i) at(T, i, i) -= mu;
    // QR of the leading m x m block by Givens rotations (T <- Q^T T = R), then T <- R Q
    std::vector<Rot> rots;
    for (int k = 0; k + 1 < m; ++k) {
      for (int i = m - 1; i > k; --i) {
        const double a = at(T, i - 1, k), b = at(T, i, k);
        if (b == 0.0) continue;
        const double r = std::hypot(a, b), cc = a / r, ss = b / r;
        for (int j = 0; j < m; ++j) {
          const double x = at(T, i - 1, j), y = at(T, i, j);
          at(T, i - 1, j) = cc * x + ss * y;
          at(T, i, j) = -ss * x + cc * y;
        }
        rots.push_back({cc, ss, i - 1, i});
      }
    }
    for (const Rot& g : rots)
      for (int row = 0; row < m; ++row) {
        const double x = at(T, row, g.i0), y = at(T, row, g.i1);
        at(T, row, g.i0) = g.c * x + g.s * y;
        at(T, row, g.i1) = -g.s * x + g.c * y;
      }
    for (int i = 0; i < m; ++i) at(T, i, i) += mu;
  }
  if (m != 0) return false;
  // eigenvectors by inverse iteration
  V.assign((size_t)n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    const double shift = E[k] + 1e-10 * nrm;
    std::vector<double> x(n);
    for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.1 * i;
    for (int it = 0; it < 4; ++it) {
      // solve (M - shift I) y = x by Gaussian elimination with partial pivoting
      std::vector<double> A(M);
      for (int i = 0; i < n; ++i) at(A, i, i) -= shift;
      std::vector<double> y(x);
      for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
          if (std::fabs(at(A, r, col)) > std::fabs(at(A, piv, col))) piv = r;
        if (at(A, piv, col) == 0.0) return false;
        if (piv != col) {
          for (int j = 0; j < n; ++j) std::swap(at(A, col, j), at(A, piv, j));
          std::swap(y[col], y[piv]);
        }
        for (int r = col + 1; r < n; ++r) {
          const double f = at(A, r, col) / at(A, col, col);
          if (f == 0.0) continue;
          for (int j = col; j < n; ++j) at(A, r, j) -= f * at(A, col, j);
          y[r] -= f * y[col];
        }
      }
      for (int r = n - 1; r >= 0; --r) {
        double v = y[r];
        for (int j = r + 1; j < n; ++j) v -= at(A, r, j) * y[j];
        y[r] = v / at(A, r, r);
      }
      double yn = 0.0;
      for (double v : y) yn += v * v;
      yn = std::sqrt(yn);
      if (!(yn > 0.0) || !std::isfinite(yn)) return false;
      for (int i = 0; i < n; ++i) x[i] = y[i] / yn;
    }
    for (int i = 0; i < n; ++i) at(V, i, k) = x[i];
  }
  // V^{-1} by Gauss-Jordan with partial pivoting
  std::vector<double> A(V);
  Vi.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) at(Vi, i, i) = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(at(A, r, col)) > std::fabs(at(A, piv, col))) piv = r;
    if (at(A, piv, col) == 0.0) return false;
    for (int j = 0; j < n; ++j) {
      std::swap(at(A, col, j), at(A, piv, j));
      std::swap(at(Vi, col, j), at(Vi, piv, j));
    }
    const double d = at(A, col, col);
    for (int j = 0; j < n; ++j) {
      at(A, col, j) /= d;
      at(Vi, col, j) /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = at(A, r, col);
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        at(A, r, j) -= f * at(A, col, j);
        at(Vi, r, j) -= f * at(Vi, col, j);
      }
    }
  }
  // check M V = V E and V V^{-1} = I
  double err = 0.0, err2 = 0.0;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double mv = 0.0, vvi = 0.0;
      for (int j = 0; j < n; ++j) {
        mv += M[(size_t)i * n + j] * V[(size_t)j * n + k];
        vvi += V[(size_t)i * n + j] * Vi[(size_t)j * n + k];
      }
      err = std::max(err, std::fabs(mv - V[(size_t)i * n + k] * E[k]));
      err2 = std::max(err2, std::fabs(vvi - (i == k ? 1.0 : 0.0)));
    }
  return err <= 1e-9 * nrm && err2 <= 1e-9;
}

}  // namespace

bool axis_eig(int n, const double* M, double* V, double* Vinv, double* E) {
  std::vector<double> m(M, M + (size_t)n * n), v, vi, e;
  if (!small_eig(n, m, v, vi, e)) return false;
  std::copy(v.begin(), v.end(), V);
  std::copy(vi.begin(), vi.end(), Vinv);
  std::copy(e.begin(), e.end(), E);
  return true;
}

int build_full_system(hps_handle* h, const double2* cdiag, cudaStream_t st) {
  FullSystem& fs = h->fs;
  const int n = h->n, ni = h->ni, nb = h->nb, n1 = h->n1, p = h->p;
  int rc = HPS_OK;
  std::vector<double2> lamq;
  if ((rc = compute_lambdas(h, cdiag, st, lamq))) return rc;
  // distinct homogenized constants
  std::map<std::pair<uint64_t, uint64_t>, int> keys;
  fs.cls.assign(h->nl, 0);
  std::vector<int> rep;
  for (int leaf = 0; leaf < h->nl; ++leaf) {
    double re = lamq[leaf].x + 0.0, im = lamq[leaf].y + 0.0;
    uint64_t a, b;
    std::memcpy(&a, &re, 8);
    std::memcpy(&b, &im, 8);
    auto it = keys.find({a, b});
    if (it == keys.end()) {
      it = keys.emplace(std::make_pair(a, b), (int)rep.size()).first;
      rep.push_back(leaf);
    }
    fs.cls[leaf] = it->second;
  }
  fs.ncls = (int)rep.size();
  const bool want64 = (h->opt.forms & HPS_FORM_FP64) != 0, want32 = (h->opt.forms & HPS_FORM_MIXED) != 0;
  const size_t per = (size_t)nb * nb;
  auto dal = [&](void** ptr, size_t bytes) -> int {
    HPS_CUDA_TRY(cudaMalloc(ptr, std::max<size_t>(bytes, 16)));
    h->bytes += std::max<size_t>(bytes, 16);
    return HPS_OK;
  };
  if (want64 && !h->opt.lean && (rc = dal((void**)&fs.Sinv64, per * fs.ncls * sizeof(double2)))) return rc;
  if (want32 && (rc = dal((void**)&fs.Sinv32, per * fs.ncls * sizeof(float2)))) return rc;
  if ((rc = dal((void**)&fs.d_cls, (size_t)h->nl * sizeof(int)))) return rc;
  HPS_CUDA_TRY(cudaMemcpyAsync(fs.d_cls, fs.cls.data(), (size_t)h->nl * sizeof(int), cudaMemcpyHostToDevice, st));
  // S~^{-1} of every distinct constant from the elimination of its homogenized leaf matrix
  {
    const int ncols = n + nb, ld = ncols;
    const long long wstride = (long long)n * ld;
    const size_t perw = (size_t)wstride * sizeof(double2);
    int nbatch = (int)std::min<size_t>((size_t)fs.ncls, std::max<size_t>(1, workspace_budget(h) / perw));
    nbatch = std::min(nbatch, 4 * h->nsm);
    double2* W = nullptr;
    int *d_status = nullptr, *d_leaves = nullptr, *d_seq = nullptr;
    HPS_CUDA_TRY(cudaMalloc(&W, perw * nbatch));
    HPS_CUDA_TRY(cudaMalloc(&d_status, sizeof(int)));
    HPS_CUDA_TRY(cudaMalloc(&d_leaves, (size_t)fs.ncls * sizeof(int)));
    HPS_CUDA_TRY(cudaMalloc(&d_seq, (size_t)fs.ncls * sizeof(int)));
    std::vector<int> seq(fs.ncls);
    for (int k = 0; k < fs.ncls; ++k) seq[k] = k;
    HPS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), st));
    HPS_CUDA_TRY(cudaMemcpyAsync(d_leaves, rep.data(), (size_t)fs.ncls * sizeof(int), cudaMemcpyHostToDevice, st));
    HPS_CUDA_TRY(cudaMemcpyAsync(d_seq, seq.data(), (size_t)fs.ncls * sizeof(int), cudaMemcpyHostToDevice, st));
    for (int k0 = 0; k0 < fs.ncls && rc == HPS_OK; k0 += nbatch) {
      const int nbt = std::min(nbatch, fs.ncls - k0);
      auto body = [&]() -> int {
        HPS_CUDA_TRY(cudaMemsetAsync(W, 0, perw * nbt, st));
        assemble_kernel<double2><<<dim3((n + 127) / 128, nbt), 128, 0, st>>>(
            W, wstride, ld, d_leaves + k0, 0, nbt, h->tables, h->tl, h->eta, nullptr, h->lambda_q, 1);
        HPS_CUDA_TRY(cudaGetLastError());
        HPS_CUDA_TRY(run_gj(W, wstride, ld, n, ncols, ni, nbt, d_status, st));
        extract_sinv_kernel<<<dim3(64, nbt), 256, 0, st>>>(W, wstride, ld, n, ni, nb, nbt, d_seq + k0, fs.Sinv64,
                                                          fs.Sinv32);
        HPS_CUDA_TRY(cudaGetLastError());
        return HPS_OK;
      };
      rc = body();
    }
    if (rc == HPS_OK) rc = check_status(d_status, st, "homogenized leaf systems");
    cudaStreamSynchronize(st);
    cudaFree(W);
    cudaFree(d_status);
    cudaFree(d_leaves);
    cudaFree(d_seq);
    if (rc) return rc;
  }
  // Algorithm 3 tables: L1 = (D~^2)[1..p-2][1..p-2] = V E V^{-1} per axis
  std::vector<double> tab(h->tl.total);
  HPS_CUDA_TRY(cudaMemcpyAsync(tab.data(), h->tables, tab.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  const size_t pa = (size_t)2 * n1 * n1 + n1;
  std::vector<double> eig(3 * pa);
  for (int axis = 0; axis < 3; ++axis) {
    std::vector<double> M((size_t)n1 * n1), V, Vi, E;
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) M[(size_t)i * n1 + j] = tab[h->tl.D2 + (size_t)axis * p * p + (i + 1) * p + (j + 1)];
    if (!small_eig(n1, M, V, Vi, E)) {
      set_error("eigen-decomposition of the 1D second-derivative block failed");
      return HPS_EBREAKDOWN;
    }
    std::copy(V.begin(), V.end(), eig.begin() + axis * pa);
    std::copy(Vi.begin(), Vi.end(), eig.begin() + axis * pa + (size_t)n1 * n1);
    std::copy(E.begin(), E.end(), eig.begin() + axis * pa + (size_t)2 * n1 * n1);
  }
  if ((rc = dal((void**)&fs.eig, eig.size() * sizeof(double)))) return rc;
  HPS_CUDA_TRY(cudaMemcpyAsync(fs.eig, eig.data(), eig.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  fs.built = true;
  return HPS_OK;
}

}  // namespace hps
