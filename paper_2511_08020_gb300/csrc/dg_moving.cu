// Moving meshes (Sec. 2: the mesh may move; Algorithm 1: the projection is
// then solved afresh because J changes with time).  Every vertex moves at a
// constant velocity, so at every volume point dx/dxi = F0 + t F1: the
// contravariant metric is a quadratic and J a cubic in t, and every face
// point's area vector a quadratic.  These kernels evaluate the geometry of
// the static curved path at a time t from those coefficients (the mass
// matrix kernel of the stage solves sits with the element transforms it
// uses, in dg_kernels.cu).
#include "dg_kernels.cuh"

namespace dgk {
namespace {

__global__ void moving_geometry_kernel(Ctx c, double* cpool, double* fgeo, double* snrm, int64_t E, int64_t nF, int n,
                                       double t) {
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
    if (snrm) {
      // each side's own outward normals (the Navier-Stokes lifting): the
      // owner's, and their negatives at the neighbour's points (a permuted
      // point set; an interpolating map only joins flat triangular faces,
      // whose normal is constant)
      double* N0 = snrm + 3 * (R.toff / 5);
      double* N1 = snrm + 3 * ((R.toff + 5 * (int64_t)n2) / 5);
#pragma unroll
      for (int d = 0; d < 3; ++d) N0[d * n2 + p] = A[d] * r;
      if (R.map >= 0) {
        const int j = c.perms[(size_t)R.map + p];
#pragma unroll
        for (int d = 0; d < 3; ++d) N1[d * n2 + j] = -A[d] * r;
      } else if (p == 0) {
        for (int k = 0; k < n2; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) N1[d * n2 + k] = -A[d] * r;
      }
    }
  }
}

}  // namespace

void launch_moving_geometry(const Ctx& c, double* cpool, double* fgeo, double* snrm, int64_t n_slots,
                            int64_t n_faces, int n, double t, int grid, cudaStream_t st) {
  moving_geometry_kernel<<<grid, 128, 0, st>>>(c, cpool, fgeo, snrm, n_slots, n_faces, n, t);
}

}  // namespace dgk
