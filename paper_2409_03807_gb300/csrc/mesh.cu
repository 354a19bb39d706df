// Rest-shape set-up kernels (Sec. 3.1 discretisation): per-tet inverse rest
// edge matrix Dm^-1 and volume V_e = det(Dm)/6, and the lumped vertex mass
// m_v = sum_{e contains v} rho V_e / 4.  FP64; run once per mesh.
#include "lsn_internal.cuh"

namespace lsn {

// Dm has the rest edges X1-X0, X2-X0, X3-X0 as columns.  dminv is stored
// structure-of-arrays: entry (a, b) of tet e at dminv[(3a+b)*ne + e].
__global__ void rest_shape_kernel(const double* __restrict__ X0,
                                  const int4* __restrict__ tets, int ne,
                                  double* __restrict__ dminv,
                                  double* __restrict__ vol, int* bad) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int4 t = tets[e];
  double D[3][3];
  int v[4] = {t.x, t.y, t.z, t.w};
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < 3; ++i) D[i][c] = X0[3 * v[c + 1] + i] - X0[3 * v[0] + i];
  // adjugate (transpose of the cofactor matrix) over the determinant
  double c00 = D[1][1] * D[2][2] - D[1][2] * D[2][1];
  double c01 = D[1][2] * D[2][0] - D[1][0] * D[2][2];
  double c02 = D[1][0] * D[2][1] - D[1][1] * D[2][0];
  double det = D[0][0] * c00 + D[0][1] * c01 + D[0][2] * c02;
  if (!(det > 0.0)) {
    atomicExch(bad, 1);
    det = 1.0;
  }
  double inv = 1.0 / det;
  double A[3][3];
  A[0][0] = c00 * inv;
  A[1][0] = c01 * inv;
  A[2][0] = c02 * inv;
  A[0][1] = (D[0][2] * D[2][1] - D[0][1] * D[2][2]) * inv;
  A[1][1] = (D[0][0] * D[2][2] - D[0][2] * D[2][0]) * inv;
  A[2][1] = (D[0][1] * D[2][0] - D[0][0] * D[2][1]) * inv;
  A[0][2] = (D[0][1] * D[1][2] - D[0][2] * D[1][1]) * inv;
  A[1][2] = (D[0][2] * D[1][0] - D[0][0] * D[1][2]) * inv;
  A[2][2] = (D[0][0] * D[1][1] - D[0][1] * D[1][0]) * inv;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) dminv[(3 * a + b) * ne + e] = A[a][b];
  vol[e] = det / 6.0;
}

// One thread per vertex, summing its incident tets in CSR order (fixed
// order, so the result does not depend on scheduling).
__global__ void lumped_mass_kernel(const int* __restrict__ adj_ptr,
                                   const int* __restrict__ adj_tet,
                                   const double* __restrict__ vol, int nv,
                                   double rho, double* __restrict__ mass) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double m = 0.0;
  for (int k = adj_ptr[v]; k < adj_ptr[v + 1]; ++k) m += rho * vol[adj_tet[k]] * 0.25;
  mass[v] = m;
}

// Displacement targets of the constrained vertices: cu = target - X0.
__global__ void constraint_disp_kernel(const int* __restrict__ cidx,
                                       const double* __restrict__ targets,
                                       const double* __restrict__ X0, int nc,
                                       double* __restrict__ cu) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nc) return;
  const int v = cidx[i / 3], k = i % 3;
  cu[i] = targets[i] - X0[3 * v + k];
}

template <typename Real>
__global__ void gather_cubature_kernel(const int4* __restrict__ tets,
                                       const double* __restrict__ dminv,
                                       const double* __restrict__ vol,
                                       const int* __restrict__ idx,
                                       const double* __restrict__ w, int s_cnt,
                                       int ne, int4* __restrict__ ctets,
                                       Real* __restrict__ cdminv,
                                       Real* __restrict__ cwv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s_cnt) return;
  int e = idx ? idx[i] : i;
  double wi = w ? w[i] : 1.0;
  ctets[i] = tets[e];
  for (int k = 0; k < 9; ++k) cdminv[k * s_cnt + i] = (Real)dminv[k * ne + e];
  cwv[i] = (Real)(wi * vol[e]);
}

template <typename Real>
__global__ void convert_kernel(const double* __restrict__ src, Real* __restrict__ dst,
                               long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < count; i += stride) dst[i] = (Real)src[i];
}

void launch_rest_shape(const double* X0, const int4* tets, int ne, double* dminv,
                       double* vol, int* bad, cudaStream_t s) {
  if (ne <= 0) return;
  rest_shape_kernel<<<(ne + 255) / 256, 256, 0, s>>>(X0, tets, ne, dminv, vol, bad);
}

void launch_lumped_mass(const int* adj_ptr, const int* adj_tet, const double* vol,
                        int nv, double rho, double* mass, cudaStream_t s) {
  if (nv <= 0) return;
  lumped_mass_kernel<<<(nv + 255) / 256, 256, 0, s>>>(adj_ptr, adj_tet, vol, nv, rho,
                                                       mass);
}

void launch_constraint_disp(const int* cidx, const double* targets, const double* X0, int nc,
                            double* cu, cudaStream_t s) {
  if (nc <= 0) return;
  constraint_disp_kernel<<<(3 * nc + 255) / 256, 256, 0, s>>>(cidx, targets, X0, nc, cu);
}

template <typename Real>
void launch_gather_cubature(const int4* tets, const double* dminv, const double* vol,
                            const int* idx, const double* w, int s_cnt, int ne,
                            int4* ctets, Real* cdminv, Real* cwv, cudaStream_t s) {
  if (s_cnt <= 0) return;
  gather_cubature_kernel<Real><<<(s_cnt + 255) / 256, 256, 0, s>>>(
      tets, dminv, vol, idx, w, s_cnt, ne, ctets, cdminv, cwv);
}

template <typename Real>
void launch_convert(const double* src, Real* dst, long long count, cudaStream_t s) {
  if (count <= 0) return;
  long long blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  convert_kernel<Real><<<(int)blocks, 256, 0, s>>>(src, dst, count);
}

template void launch_gather_cubature<float>(const int4*, const double*, const double*,
                                            const int*, const double*, int, int, int4*,
                                            float*, float*, cudaStream_t);
template void launch_gather_cubature<double>(const int4*, const double*, const double*,
                                             const int*, const double*, int, int, int4*,
                                             double*, double*, cudaStream_t);
template void launch_convert<float>(const double*, float*, long long, cudaStream_t);
template void launch_convert<double>(const double*, double*, long long, cudaStream_t);

}  // namespace lsn
