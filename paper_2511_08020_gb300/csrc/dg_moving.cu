// Moving meshes (Sec. 2: the mesh may move; Algorithm 1: the projection is
// then solved afresh because J changes with time).  Every vertex moves at a
// constant velocity, so at every volume point dx/dxi = F0 + t F1: the
// contravariant metric is a quadratic and J a cubic in t, and every face
// point's area vector a quadratic.  These kernels evaluate the geometry of
// the static curved path at a time t from those coefficients, and apply or
// solve the element mass matrix M^ = V^T diag(w J^) V with J^ = sum_k tau_k
// J_k, tau_k the LSERK stage value of t^k (the discrete geometric
// conservation law: a constant state stays constant to rounding).
#include "dg_kernels.cuh"

namespace dgk {
namespace {

constexpr int kMassThreads = 128;

__global__ void moving_geometry_kernel(Ctx c, double* cpool, double* fgeo, int64_t E, int64_t nF, int n, double t) {
  for (int64_t s = blockIdx.x; s < E; s += gridDim.x) {
    const TypeTab& T = c.tabs[c.slot_tab[s]];
    const int nQ = T.nQ;
    const double* m = c.mpool + c.slot_moff[s];
    double* cb = cpool + c.slot_coff[s];
    for (int q = threadIdx.x; q < nQ; q += blockDim.x) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
        cb[i * nQ + q] = fma(t, fma(t, m[(18 + i) * nQ + q], m[(9 + i) * nQ + q]), m[i * nQ + q]);
      const double J = fma(t, fma(t, fma(t, m[30 * nQ + q], m[29 * nQ + q]), m[28 * nQ + q]), m[27 * nQ + q]);
      cb[9 * nQ + q] = J;
      cb[10 * nQ + q] = 1.0 / J;
      if (!(J > 0.0)) atomicOr(c.status, 4u);
    }
  }
  const int n2 = n * n;
  const int64_t items = nF * n2;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < items; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = w / n2;
    const int p = (int)(w - f * n2);
    const FaceRec& R = c.faces[f];
    if (R.cgeo < 0) continue;
    const double* a = c.fmot + 3 * (int64_t)R.cgeo;
    double A[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) A[d] = fma(t, fma(t, a[(6 + d) * n2 + p], a[(3 + d) * n2 + p]), a[d * n2 + p]);
    const double S = sqrt(fma(A[0], A[0], fma(A[1], A[1], A[2] * A[2])));   // w S (the weight is in A)
    double* g = fgeo + R.cgeo;
    const double r = 1.0 / S;
#pragma unroll
    for (int d = 0; d < 3; ++d) g[d * n2 + p] = A[d] * r;
    g[3 * n2 + p] = S;
    if (!(S > 0.0)) atomicOr(c.status, 4u);
  }
}

// One block per element at a time.  Hexahedra (scaled nodal storage
// s = W^{1/2} V q, V square with V^T W V = I): M^ q in that storage is
// J^ s pointwise.  Prisms and pyramids: M^ assembled in shared memory, then
// either applied or factored (Cholesky, lower, in place) and solved for the
// five variables.
__global__ void __launch_bounds__(kMassThreads) moving_mass_kernel(Ctx c, int64_t E, const double* in, double* out,
                                                                   double t0, double t1, double t2, double t3,
                                                                   int weight) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int64_t s = blockIdx.x; s < E; s += gridDim.x) {
    const TypeTab& T = c.tabs[c.slot_tab[s]];
    const int nQ = T.nQ, nM = T.nM;
    const int64_t qoff = c.slot_qoff[s];
    const double* m = c.mpool + c.slot_moff[s];
    if (T.type == HEX) {
      for (int w = tid; w < 5 * nQ; w += bd) {
        const int q = w % nQ;
        const double J = fma(t3, m[30 * nQ + q], fma(t2, m[29 * nQ + q], fma(t1, m[28 * nQ + q], t0 * m[27 * nQ + q])));
        const double x = in[qoff + w];
        out[qoff + w] = weight ? x * J : x / J;
      }
      continue;   // block-uniform: every thread takes the same branch
    }
    double* Mh = sm;
    double* b = sm + nM * nM;
    const double* Mk = m + 34 * nQ;
    const int nn = nM * nM;
    for (int w = tid; w < nn; w += bd)
      Mh[w] = fma(t3, Mk[3 * nn + w], fma(t2, Mk[2 * nn + w], fma(t1, Mk[nn + w], t0 * Mk[w])));
    for (int w = tid; w < 5 * nM; w += bd) b[w] = in[qoff + w];
    __syncthreads();
    if (weight) {
      for (int w = tid; w < 5 * nM; w += bd) {
        const int v = w / nM, a = w - v * nM;
        const double* row = Mh + a * nM;
        const double* x = b + v * nM;
        double acc = 0.0;
        for (int k = 0; k < nM; ++k) acc = fma(row[k], x[k], acc);
        out[qoff + w] = acc;
      }
      __syncthreads();
      continue;
    }
    // Cholesky M^ = L L^T, column by column (right-looking)
    for (int j = 0; j < nM; ++j) {
      const double d = sqrt(Mh[j * nM + j]);
      const double rd = 1.0 / d;
      for (int i = j + 1 + tid; i < nM; i += bd) Mh[i * nM + j] *= rd;
      __syncthreads();
      if (tid == 0) Mh[j * nM + j] = d;
      const int r = nM - j - 1;
      for (int w = tid; w < r * r; w += bd) {
        const int ii = w / r, kk = w - ii * r;
        if (kk > ii) continue;
        const int i = j + 1 + ii, k = j + 1 + kk;
        Mh[i * nM + k] = fma(-Mh[i * nM + j], Mh[k * nM + j], Mh[i * nM + k]);
      }
      __syncthreads();
    }
    // L y = b, then L^T x = y (the five variables side by side)
    for (int j = 0; j < nM; ++j) {
      if (tid < 5) b[tid * nM + j] /= Mh[j * nM + j];
      __syncthreads();
      const int r = nM - j - 1;
      for (int w = tid; w < 5 * r; w += bd) {
        const int v = w / r, i = j + 1 + (w - v * r);
        b[v * nM + i] = fma(-Mh[i * nM + j], b[v * nM + j], b[v * nM + i]);
      }
      __syncthreads();
    }
    for (int j = nM - 1; j >= 0; --j) {
      if (tid < 5) b[tid * nM + j] /= Mh[j * nM + j];
      __syncthreads();
      for (int w = tid; w < 5 * j; w += bd) {
        const int v = w / j, i = w - v * j;
        b[v * nM + i] = fma(-Mh[j * nM + i], b[v * nM + j], b[v * nM + i]);
      }
      __syncthreads();
    }
    for (int w = tid; w < 5 * nM; w += bd) out[qoff + w] = b[w];
    __syncthreads();
  }
}

}  // namespace

void launch_moving_geometry(const Ctx& c, double* cpool, double* fgeo, int64_t n_slots, int64_t n_faces, int n,
                            double t, int grid, cudaStream_t st) {
  moving_geometry_kernel<<<grid, 128, 0, st>>>(c, cpool, fgeo, n_slots, n_faces, n, t);
}

cudaError_t launch_moving_mass(const Ctx& c, int64_t n_slots, const double* in, double* out, const double* tau,
                               int weight, int max_nM, int grid, cudaStream_t st) {
  const size_t bytes = max_nM > 0 ? sizeof(double) * ((size_t)max_nM * max_nM + 5 * (size_t)max_nM) : 0;
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(moving_mass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  moving_mass_kernel<<<grid, kMassThreads, bytes, st>>>(c, n_slots, in, out, tau[0], tau[1], tau[2], tau[3], weight);
  return cudaGetLastError();
}

}  // namespace dgk
