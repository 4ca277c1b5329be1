// The paper's own iterative path on the global system (Sec. 3-4): unknowns are
// the values of u at every node of every leaf (n = n_i + n_b per leaf, the
// leaf's interior nodes x fastest, then its six faces' n1 x n1 Chebyshev
// nodes).
//
//  * apply    y = A u, A of eq. (2x2): per leaf the interior rows
//             -(D_x^2 + D_y^2 + D_z^2) u - C u along the three lines through
//             each interior node (eq. (leafmat), the mode products of
//             Algorithm 1; each grid line ends on two face nodes), the face rows
//             F u = N u + i eta u, and on a face shared with beta the
//             neighbour's outgoing data G^beta u^beta = N^beta u^beta - i eta u^beta
//             at the same points (Algorithm 2, eq. (inter)).
//  * precond  z = A~^{-1} r leaf by leaf (Sec. 4, eq. (block_pc), Algorithm 4):
//             y = A~_ii^{-1} r_i by Algorithm 3 (mode products with V^{-1},
//             division by -(E_x + E_y + E_z) - lambda, mode products with V),
//             z_b = S~^{-1} (r_b - F_bi y), z_i = A~_ii^{-1} (r_i - A_ib z_b);
//             S~^{-1} = (A~^{-1})_bb per distinct (binned) lambda from setup.
//
// One CTA per (right-hand side, leaf); the leaf's vector is staged in shared
// memory; neighbour values needed by the coupling rows are read from global
// memory (L2).  R is the arithmetic type (float for the mixed form, double for
// the FP64 form and the residual).
#include <algorithm>

#include "common.cuh"
#include "hps_internal.h"

namespace hps {

namespace {

constexpr int kFT = 256;

template <class R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

template <class C, class R> __device__ __forceinline__ void rfma(C& acc, R s, C a) {
  acc.x = fma(s, a.x, acc.x);
  acc.y = fma(s, a.y, acc.y);
}
// i * s * a
template <class C, class R> __device__ __forceinline__ C imul(C a, R s) {
  C o;
  o.x = -a.y * s;
  o.y = a.x * s;
  return o;
}

// Local index of grid node (i, j, k), 0 <= i, j, k < p, not on an edge or corner.
__device__ __forceinline__ int node(int i, int j, int k, int p, int n1, int ni) {
  const int last = p - 1;
  const bool bi = (i == 0 || i == last), bj = (j == 0 || j == last), bk = (k == 0 || k == last);
  if (!bi && !bj && !bk) return (i - 1) + n1 * ((j - 1) + n1 * (k - 1));
  int face, a, b;
  if (bi) { face = (i == 0) ? 0 : 1; a = j; b = k; }
  else if (bj) { face = (j == 0) ? 2 : 3; a = i; b = k; }
  else { face = (k == 0) ? 4 : 5; a = i; b = j; }
  return ni + face * n1 * n1 + (a - 1) + n1 * (b - 1);
}

struct FullGeom {
  int p, n1, ni, nb, n, nl;
  GridDims g;
};

// (i, j, k) of face node jb of a leaf: face = jb / n1^2, in-face (a, b), first axis fastest
__device__ __forceinline__ void face_point(int jb, int p, int n1, int& face, int (&pt)[3]) {
  face = jb / (n1 * n1);
  const int rem = jb % (n1 * n1);
  const int a = rem % n1 + 1, b = rem / n1 + 1;
  const int axis = face >> 1;
  pt[axis] = (face & 1) ? p - 1 : 0;
  pt[axis == 0 ? 1 : 0] = a;
  pt[axis == 2 ? 1 : 2] = b;
}

struct FullApplyArgs {
  FullGeom G;
  const double* D;   // 3 x p x p, scaled to the leaf widths
  const double* D2;  // squares of D
  const double2* cdiag;
  double eta;
  const void* u;
  void* y;
  const double2* b;  // residual mode: y = b - A u
  long long nu;      // values per right-hand side
  int nrhs;
  const int* gate;   // while a GMRES cycle is replayed: 0 = return at once
};

template <class R, class TIN, class TOUT>
__global__ void __launch_bounds__(kFT) full_apply_kernel(FullApplyArgs a) {
  if (a.gate && *a.gate == 0) return;
  using C = typename Cx<R>::T;
  const int p = a.G.p, n1 = a.G.n1, ni = a.G.ni, n = a.G.n;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* us = reinterpret_cast<C*>(smraw);
  R* sD = reinterpret_cast<R*>(us + n);
  R* sD2 = sD + 3 * p * p;
  for (int t = threadIdx.x; t < 3 * p * p; t += kFT) {
    sD[t] = (R)a.D[t];
    sD2[t] = (R)a.D2[t];
  }
  const R eta = (R)a.eta;
  const TIN* uin = reinterpret_cast<const TIN*>(a.u);
  TOUT* yo = reinterpret_cast<TOUT*>(a.y);
  const long long items = (long long)a.G.nl * a.nrhs;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int rhs = (int)(item / a.G.nl), leaf = (int)(item % a.G.nl);
    const long long base = rhs * a.nu + (long long)leaf * n;
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += kFT) us[t] = cvt<C>(uin[base + t]);
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += kFT) {
      C val = czero<C>();
      if (r < ni) {
        const int i = r % n1 + 1, j = (r / n1) % n1 + 1, k = r / (n1 * n1) + 1;
        for (int m = 0; m < p; ++m) {
          rfma(val, sD2[0 * p * p + i * p + m], us[node(m, j, k, p, n1, ni)]);
          rfma(val, sD2[1 * p * p + j * p + m], us[node(i, m, k, p, n1, ni)]);
          rfma(val, sD2[2 * p * p + k * p + m], us[node(i, j, m, p, n1, ni)]);
        }
        const C cu = cmul(cvt<C>(a.cdiag[(long long)leaf * ni + r]), us[r]);
        val.x = -val.x - cu.x;
        val.y = -val.y - cu.y;
      } else {
        int face, pt[3];
        face_point(r - ni, p, n1, face, pt);
        const int axis = face >> 1, e = pt[axis];
        const R sg = (face & 1) ? (R)1 : (R)-1;
        for (int m = 0; m < p; ++m) {
          int q3[3] = {pt[0], pt[1], pt[2]};
          q3[axis] = m;
          rfma(val, sg * sD[axis * p * p + e * p + m], us[node(q3[0], q3[1], q3[2], p, n1, ni)]);
        }
        val = cadd(val, imul(us[r], eta));
        const int nbr = a.G.g.neighbor(leaf, face);
        if (nbr >= 0) {
          // beta's outgoing data on its opposite face, at the same point
          const long long nb_base = rhs * a.nu + (long long)nbr * n;
          const int eb = p - 1 - e;
          const R sgb = -sg;
          C gb = czero<C>();
          for (int m = 0; m < p; ++m) {
            int q3[3] = {pt[0], pt[1], pt[2]};
            q3[axis] = m;
            rfma(gb, sgb * sD[axis * p * p + eb * p + m], cvt<C>(uin[nb_base + node(q3[0], q3[1], q3[2], p, n1, ni)]));
          }
          int qf[3] = {pt[0], pt[1], pt[2]};
          qf[axis] = eb;
          const C uf = cvt<C>(uin[nb_base + node(qf[0], qf[1], qf[2], p, n1, ni)]);
          gb = csub(gb, imul(uf, eta));
          val = cadd(val, gb);
        }
      }
      if (a.b) {
        const double2 bv = a.b[base + r];
        yo[base + r] = cvt<TOUT>(make_double2(bv.x - (double)val.x, bv.y - (double)val.y));
      } else {
        yo[base + r] = cvt<TOUT>(val);
      }
    }
  }
}

// Algorithm 3 on the block's shared buffers: out = A~_ii^{-1} in (complex,
// n1^3 values, x fastest).  tmp is a second buffer of the same size; in is
// preserved.  Tables per axis: V, V^{-1} (n1 x n1 row-major) and E (n1).
template <class R, class C>
__device__ void alg3_inverse(const C* in, C* out, C* tmp, const R* eig, int n1, C lam) {
  const int ni = n1 * n1 * n1;
  const int pa = 2 * n1 * n1 + n1;
  // mode products with V^{-1} along x, y, z: in -> tmp -> out -> tmp
  const C* src = in;
  C* bufs[3] = {tmp, out, tmp};
  for (int axis = 0; axis < 3; ++axis) {
    const R* Vi = eig + axis * pa + n1 * n1;
    C* dst = bufs[axis];
    for (int t = threadIdx.x; t < ni; t += blockDim.x) {
      int c3[3] = {t % n1, (t / n1) % n1, t / (n1 * n1)};
      const int row = c3[axis];
      C acc = czero<C>();
      for (int m = 0; m < n1; ++m) {
        c3[axis] = m;
        rfma(acc, Vi[row * n1 + m], src[c3[0] + n1 * (c3[1] + n1 * c3[2])]);
      }
      dst[t] = acc;
    }
    __syncthreads();
    src = dst;
  }
  // divide by -(E_x + E_y + E_z) - lambda
  for (int t = threadIdx.x; t < ni; t += blockDim.x) {
    const int i = t % n1, j = (t / n1) % n1, k = t / (n1 * n1);
    const R ed = eig[0 * pa + 2 * n1 * n1 + i] + eig[1 * pa + 2 * n1 * n1 + j] + eig[2 * pa + 2 * n1 * n1 + k];
    C d;
    d.x = -ed - lam.x;
    d.y = -lam.y;
    tmp[t] = cmul(tmp[t], cinv(d));
  }
  __syncthreads();
  // mode products with V along x, y, z: tmp -> out -> tmp -> out
  src = tmp;
  C* bufs2[3] = {out, tmp, out};
  for (int axis = 0; axis < 3; ++axis) {
    const R* V = eig + axis * pa;
    C* dst = bufs2[axis];
    for (int t = threadIdx.x; t < ni; t += blockDim.x) {
      int c3[3] = {t % n1, (t / n1) % n1, t / (n1 * n1)};
      const int row = c3[axis];
      C acc = czero<C>();
      for (int m = 0; m < n1; ++m) {
        c3[axis] = m;
        rfma(acc, V[row * n1 + m], src[c3[0] + n1 * (c3[1] + n1 * c3[2])]);
      }
      dst[t] = acc;
    }
    __syncthreads();
    src = dst;
  }
}

struct FullPrecArgs {
  FullGeom G;
  const double* D;
  const double* D2;
  const double* eig;       // 3 x (2 n1^2 + n1)
  const double2* lam;      // binned lambda per leaf
  const int* cls;          // class of each leaf
  const void* S;           // S~^{-1} per class, nb x nb row-major
  const void* r;
  void* z;
  long long nu;
  int nrhs;
  const int* gate;   // as in FullApplyArgs
};

template <class R, class TS, class TIN, class TOUT>
__global__ void __launch_bounds__(kFT) full_precond_kernel(FullPrecArgs a) {
  if (a.gate && *a.gate == 0) return;
  using C = typename Cx<R>::T;
  const int p = a.G.p, n1 = a.G.n1, ni = a.G.ni, nb = a.G.nb, n = a.G.n;
  const int pa = 2 * n1 * n1 + n1;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* rs = reinterpret_cast<C*>(smraw);  // n: r
  C* y = rs + n;                        // ni
  C* t1 = y + ni;                       // ni
  C* t2 = t1 + ni;                      // ni
  C* wb = t2 + ni;                      // nb
  C* zb = wb + nb;                      // nb
  R* sD = reinterpret_cast<R*>(zb + nb);
  R* sD2 = sD + 3 * p * p;
  R* seig = sD2 + 3 * p * p;
  for (int t = threadIdx.x; t < 3 * p * p; t += kFT) {
    sD[t] = (R)a.D[t];
    sD2[t] = (R)a.D2[t];
  }
  for (int t = threadIdx.x; t < 3 * pa; t += kFT) seig[t] = (R)a.eig[t];
  const TIN* rin = reinterpret_cast<const TIN*>(a.r);
  TOUT* zo = reinterpret_cast<TOUT*>(a.z);
  const TS* S = reinterpret_cast<const TS*>(a.S);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long items = (long long)a.G.nl * a.nrhs;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int rhs = (int)(item / a.G.nl), leaf = (int)(item % a.G.nl);
    const long long base = rhs * a.nu + (long long)leaf * n;
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += kFT) rs[t] = cvt<C>(rin[base + t]);
    __syncthreads();
    const C lam = cvt<C>(a.lam[leaf]);
    // y = A~_ii^{-1} r_i
    alg3_inverse<R, C>(rs, y, t1, seig, n1, lam);
    // w_b = r_b - F_bi y (interior points of the line through each face node)
    for (int jb = threadIdx.x; jb < nb; jb += kFT) {
      int face, pt[3];
      face_point(jb, p, n1, face, pt);
      const int axis = face >> 1, e = pt[axis];
      const R sg = (face & 1) ? (R)1 : (R)-1;
      C acc = czero<C>();
      for (int m = 1; m < p - 1; ++m) {
        int q3[3] = {pt[0], pt[1], pt[2]};
        q3[axis] = m;
        rfma(acc, sg * sD[axis * p * p + e * p + m], y[(q3[0] - 1) + n1 * ((q3[1] - 1) + n1 * (q3[2] - 1))]);
      }
      wb[jb] = csub(rs[ni + jb], acc);
    }
    __syncthreads();
    // z_b = S~^{-1} w_b (one warp per row, lanes over columns; a thread per row on a
    // transposed S~^{-1} was measured slower: its 384-term dependent chain per thread)
    const TS* Sk = S + (long long)a.cls[leaf] * nb * nb;
    for (int row = warp; row < nb; row += kFT / 32) {
      C acc = czero<C>();
      for (int c = lane; c < nb; c += 32) cfma(acc, cvt<C>(Sk[(long long)row * nb + c]), wb[c]);
      acc.x = warp_sum(acc.x);
      acc.y = warp_sum(acc.y);
      if (lane == 0) zb[row] = acc;
    }
    __syncthreads();
    // t2 = r_i - A_ib z_b: A_ib holds -D2 at the line ends (face nodes)
    for (int t = threadIdx.x; t < ni; t += kFT) {
      const int c3[3] = {t % n1 + 1, (t / n1) % n1 + 1, t / (n1 * n1) + 1};
      C v = rs[t];
      for (int axis = 0; axis < 3; ++axis) {
        for (int end = 0; end < 2; ++end) {
          const int m = end ? p - 1 : 0;
          int q3[3] = {c3[0], c3[1], c3[2]};
          q3[axis] = m;
          rfma(v, sD2[axis * p * p + c3[axis] * p + m], zb[node(q3[0], q3[1], q3[2], p, n1, ni) - ni]);
        }
      }
      t2[t] = v;
    }
    __syncthreads();
    // z_i = A~_ii^{-1} t2 (result in y; t1 is scratch)
    alg3_inverse<R, C>(t2, y, t1, seig, n1, lam);
    for (int t = threadIdx.x; t < n; t += kFT) zo[base + t] = cvt<TOUT>(t < ni ? y[t] : zb[t - ni]);
  }
}

// b = [s at interior nodes; P^{-1} t on faces on the boundary of (0,1)^3; 0 on
// shared faces], P^{-1} F = Qi F Qi^T per face (Gauss points to Chebyshev nodes).
__global__ void full_rhs_kernel(FullGeom G, const double* Qi, int q, const double2* s, const double2* t, double2* b,
                                long long nu, long long nint, long long nf, int nrhs) {
  const int n = G.n, ni = G.ni, q2 = q * q;
  const long long total = (long long)nrhs * nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(e / nu);
    const long long w = e % nu;
    const int leaf = (int)(w / n), r = (int)(w % n);
    double2 v = make_double2(0.0, 0.0);
    if (r < ni) {
      if (s) v = s[rhs * nint + (long long)leaf * ni + r];
    } else if (t) {
      const int jb = r - ni, face = jb / q2, rem = jb % q2, a = rem % q, bb = rem / q;
      if (G.g.neighbor(leaf, face) < 0) {
        const double2* tf = t + rhs * nf + (long long)leaf * 6 * q2 + (long long)face * q2;
        for (int j2 = 0; j2 < q; ++j2)
          for (int j1 = 0; j1 < q; ++j1) {
            const double w2 = Qi[bb * q + j2] * Qi[a * q + j1];
            const double2 tv = tf[j2 * q + j1];
            v.x += w2 * tv.x;
            v.y += w2 * tv.y;
          }
      }
    }
    b[e] = v;
  }
}

FullGeom full_geom(const hps_handle* h) {
  FullGeom G;
  G.p = h->p;
  G.n1 = h->n1;
  G.ni = h->ni;
  G.nb = h->nb;
  G.n = h->n;
  G.nl = h->nl;
  G.g = GridDims{h->nx, h->ny, h->nz};
  return G;
}

template <class R, class TIN, class TOUT>
cudaError_t full_apply_t(const hps_handle* h, const void* u, void* y, const double2* b, int nrhs, cudaStream_t st) {
  using C = typename Cx<R>::T;
  FullApplyArgs a;
  a.G = full_geom(h);
  a.D = h->tables + h->tl.D;
  a.D2 = h->tables + h->tl.D2;
  a.cdiag = h->cdiag;
  a.eta = h->eta;
  a.u = u;
  a.y = y;
  a.b = b;
  a.nu = (long long)h->nl * h->n;
  a.nrhs = nrhs;
  a.gate = h->gate;
  const size_t smem = (size_t)h->n * sizeof(C) + (size_t)6 * h->p * h->p * sizeof(R);
  auto kern = full_apply_kernel<R, TIN, TOUT>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kFT, smem);
  if (e != cudaSuccess) return e;
  const long long items = (long long)h->nl * nrhs;
  const int grid = (int)std::min<long long>(items, (long long)h->nsm * std::max(occ, 1));
  kern<<<grid, kFT, smem, st>>>(a);
  ++h->prof.launches;
  return cudaGetLastError();
}

template <class R, class TS, class TIN, class TOUT>
cudaError_t full_precond_t(const hps_handle* h, const TS* S, const void* r, void* z, int nrhs, cudaStream_t st) {
  using C = typename Cx<R>::T;
  if (!h->fs.built || !S) return cudaErrorInvalidValue;
  FullPrecArgs a;
  a.G = full_geom(h);
  a.D = h->tables + h->tl.D;
  a.D2 = h->tables + h->tl.D2;
  a.eig = h->fs.eig;
  a.lam = h->lambda_q;
  a.cls = h->fs.d_cls;
  a.S = S;
  a.r = r;
  a.z = z;
  a.nu = (long long)h->nl * h->n;
  a.nrhs = nrhs;
  a.gate = h->gate;
  const int pa = 2 * h->n1 * h->n1 + h->n1;
  const size_t smem =
      (size_t)(h->n + 3 * h->ni + 2 * h->nb) * sizeof(C) + (size_t)(6 * h->p * h->p + 3 * pa) * sizeof(R);
  auto kern = full_precond_kernel<R, TS, TIN, TOUT>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kFT, smem);
  if (e != cudaSuccess) return e;
  const long long items = (long long)h->nl * nrhs;
  const int grid = (int)std::min<long long>(items, (long long)h->nsm * std::max(occ, 1));
  kern<<<grid, kFT, smem, st>>>(a);
  ++h->prof.launches;
  return cudaGetLastError();
}

}  // namespace

// y = A u (global system), or y = b - A u when b is given (complex double only).
// fp64: complex-double arithmetic; otherwise complex-float arithmetic.
cudaError_t launch_full_apply(const hps_handle* h, bool fp64, VType tin, const void* u, VType tout, void* y,
                              const double2* b, int nrhs, cudaStream_t st) {
  if (b && !(fp64 && tin == VType::C128 && tout == VType::C128)) return cudaErrorInvalidValue;
  if (fp64) {
    if (tin == VType::C128 && tout == VType::C128) return full_apply_t<double, double2, double2>(h, u, y, b, nrhs, st);
    return cudaErrorInvalidValue;
  }
  if (tin == VType::C64 && tout == VType::DF) return full_apply_t<float, float2, float4>(h, u, y, b, nrhs, st);
  if (tin == VType::DF && tout == VType::DF) return full_apply_t<float, float4, float4>(h, u, y, b, nrhs, st);
  if (tin == VType::C64 && tout == VType::C64) return full_apply_t<float, float2, float2>(h, u, y, b, nrhs, st);
  return cudaErrorInvalidValue;
}

// z = A~^{-1} r leaf by leaf (block-Jacobi of Sec. 4 on the global system).
cudaError_t launch_full_precond(const hps_handle* h, bool fp64, VType tin, const void* r, VType tout, void* z,
                                int nrhs, cudaStream_t st) {
  if (fp64) {
    if (tin == VType::C128 && tout == VType::C128)
      return full_precond_t<double, double2, double2, double2>(h, h->fs.Sinv64, r, z, nrhs, st);
    return cudaErrorInvalidValue;
  }
  if (tout != VType::C64) return cudaErrorInvalidValue;
  if (tin == VType::DF) return full_precond_t<float, float2, float4, float2>(h, h->fs.Sinv32, r, z, nrhs, st);
  if (tin == VType::C128) return full_precond_t<float, float2, double2, float2>(h, h->fs.Sinv32, r, z, nrhs, st);
  if (tin == VType::C64) return full_precond_t<float, float2, float2, float2>(h, h->fs.Sinv32, r, z, nrhs, st);
  return cudaErrorInvalidValue;
}

// The paper's iterative method on the global system: restarted GMRES with the
// leaf block-Jacobi preconditioner (right preconditioning, FP64 residual each
// restart).  s: nrhs interior vectors or NULL, t: nrhs face vectors at Gauss
// points or NULL, u: nrhs global vectors (device).
int full_solve(hps_handle* h, int form, bool use_precond, const double2* s, const double2* t, int nrhs, double tol,
               double2* u, hps_solve_info* info, cudaStream_t st, SolveFlags fl) {
  const bool mixed = (form == HPS_FORM_MIXED);
  const long long nu = (long long)h->nl * h->n;
  int rc = krylov_alloc(h, nrhs, nu);
  if (rc) return rc;
  const FullGeom G = full_geom(h);
  full_rhs_kernel<<<4 * h->nsm, 256, 0, st>>>(G, h->tables + h->tl.Qi, h->q, s, t, h->ks.b, nu, h->nint, h->nf, nrhs);
  HPS_CUDA_TRY(cudaGetLastError());
  ++h->prof.launches;
  GmresOps ops;
  ops.n = nu;
  ops.pc = use_precond && h->fs.built;
  ops.apply = [h, mixed](VType tin, const void* in, VType tout, void* out, int nr, cudaStream_t s2) {
    cudaEvent_t ev = h->prof.begin(s2);
    cudaError_t e = launch_full_apply(h, !mixed, tin, in, tout, out, nullptr, nr, s2);
    h->prof.end(HPS_PHASE_APPLY, ev, s2);
    return e;
  };
  ops.precond = [h, mixed](VType tin, const void* in, VType tout, void* out, int nr, cudaStream_t s2) {
    cudaEvent_t ev = h->prof.begin(s2);
    cudaError_t e = launch_full_precond(h, !mixed, tin, in, tout, out, nr, s2);
    h->prof.end(HPS_PHASE_PRECOND_K, ev, s2);
    return e;
  };
  ops.residual = [h](const double2* x, const double2* b, double2* r, int nr, cudaStream_t s2) {
    cudaEvent_t ev = h->prof.begin(s2);
    cudaError_t e = launch_full_apply(h, true, VType::C128, x, VType::C128, r, b, nr, s2);
    h->prof.end(HPS_PHASE_RESIDUAL, ev, s2);
    return e;
  };
  ops.id = 1;
  return gmres_core(h, ops, mixed, h->ks.b, u, nrhs, tol, info, st, fl);
}

}  // namespace hps
