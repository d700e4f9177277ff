// axes.cu - spaces whose Shen axis is not axis 0 (or whose R2C axis is not the last one): the
// axes option of the paper's TensorProductSpace (Sec. 4: TensorProductSpace(comm, (K1, K0),
// axes=(1, 0)), the Dirichlet basis along the second axis).
//
// Every transform and solve of the library works on the canonical layout: the polynomial axis
// first, the C2C axes in their given order, the R2C axis last.  A space created with another axis
// order is a view of a canonical space: its arrays are axis permutations of the canonical ones.
// The transforms along the axes are the same in any order (they act on different indices), so
// each call permutes its input into a canonical workspace, runs the canonical call and permutes
// the result back.  The permutation is one pass over the array (k_permute: one output element
// per thread, consecutive threads on consecutive output elements, the reads strided).
#include <algorithm>
#include <cstring>

#include "space_internal.cuh"

namespace sgm {
namespace {

struct Shape3 {
  long n[3];      // extents of the input array (unused trailing axes 1)
  int to_out[3];  // output axis that input axis d becomes
  long on[3];     // extents of the output array
};

template <typename E>
__global__ void __launch_bounds__(256) k_permute(const E* __restrict__ in, E* __restrict__ out, long total,
                                                 const __grid_constant__ Shape3 sh) {
  for (long o = (long)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (long)gridDim.x * blockDim.x) {
    long oc[3];
    long r = o;
    oc[2] = r % sh.on[2];
    r /= sh.on[2];
    oc[1] = r % sh.on[1];
    oc[0] = r / sh.on[1];
    const long i0 = oc[sh.to_out[0]], i1 = oc[sh.to_out[1]], i2 = oc[sh.to_out[2]];
    out[o] = in[(i0 * sh.n[1] + i1) * sh.n[2] + i2];
  }
}

// out = in with input axis d moved to output axis to_out[d]; elem bytes 4, 8 or 16
int permute(const void* in, void* out, int ndim, const int64_t* in_shape, const int* to_out, size_t elem,
            cudaStream_t st) {
  Shape3 sh;
  for (int d = 0; d < 3; ++d) {
    sh.n[d] = d < ndim ? (long)in_shape[d] : 1;
    sh.to_out[d] = d < ndim ? to_out[d] : d;
    sh.on[d] = 1;
  }
  for (int d = 0; d < ndim; ++d) sh.on[to_out[d]] = sh.n[d];
  const long total = sh.n[0] * sh.n[1] * sh.n[2];
  if (total == 0) return SGM_OK;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<long>((total + 255) / 256, (long)sms * 8);
  if (elem == 4) k_permute<int><<<grid, 256, 0, st>>>((const int*)in, (int*)out, total, sh);
  else if (elem == 8) k_permute<int2><<<grid, 256, 0, st>>>((const int2*)in, (int2*)out, total, sh);
  else k_permute<int4><<<grid, 256, 0, st>>>((const int4*)in, (int4*)out, total, sh);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "axis permutation: %s", cudaGetErrorString(e));
  return SGM_OK;
}

bool polynomial_kind(int k) {
  return k == SGM_CHEBYSHEV || k == SGM_SHEN_DIRICHLET || k == SGM_SHEN_BIHARMONIC || k == SGM_SHEN_NEUMANN ||
         k == SGM_LEGENDRE || k == SGM_LEGENDRE_DIRICHLET || k == SGM_LEGENDRE_BIHARMONIC;
}

}  // namespace

bool canonical_axes(int ndim, const int* kinds) {
  for (int d = 0; d < ndim; ++d) {
    if (d > 0 && polynomial_kind(kinds[d])) return false;
    if (kinds[d] == SGM_FOURIER_R2C && d != ndim - 1) return false;
  }
  return true;
}

int permuted_create(sgm_space** out, int ndim, const int* kinds, const int64_t* n, const double* domain, int precision) {
  int npoly = 0, nr2c = 0;
  for (int d = 0; d < ndim; ++d) {
    if (kinds[d] < SGM_CHEBYSHEV || kinds[d] > SGM_SHEN_NEUMANN)
      return set_error(SGM_ERR_ARG, "axis %d: unknown basis kind %d", d, kinds[d]);
    npoly += polynomial_kind(kinds[d]);
    nr2c += kinds[d] == SGM_FOURIER_R2C;
  }
  if (npoly > 1) return set_error(SGM_ERR_SIZE, "at most one Chebyshev or Legendre axis");
  if (nr2c > 1) return set_error(SGM_ERR_SIZE, "at most one R2C axis");
  // canonical order: the polynomial axis, the C2C axes in their order, the R2C axis
  int order[3], m = 0;
  for (int d = 0; d < ndim; ++d)
    if (polynomial_kind(kinds[d])) order[m++] = d;
  for (int d = 0; d < ndim; ++d)
    if (kinds[d] == SGM_FOURIER_C2C) order[m++] = d;
  for (int d = 0; d < ndim; ++d)
    if (kinds[d] == SGM_FOURIER_R2C) order[m++] = d;
  int ck[3];
  int64_t cn[3];
  double cdom[6];
  for (int c = 0; c < ndim; ++c) {
    ck[c] = kinds[order[c]];
    cn[c] = n[order[c]];
    if (domain) {
      cdom[2 * c] = domain[2 * order[c]];
      cdom[2 * c + 1] = domain[2 * order[c] + 1];
    }
  }
  sgm_space* inner = nullptr;
  const int st = sgm_space_create(&inner, ndim, ck, cn, domain ? cdom : nullptr, precision);
  if (st != SGM_OK) return st;
  sgm_space* s = new (std::nothrow) sgm_space;
  if (!s) {
    sgm_space_destroy(inner);
    return set_error(SGM_ERR_ALLOC, "host allocation failed");
  }
  s->device = inner->device;
  s->ndim = ndim;
  s->prec = inner->prec;
  s->cheb = inner->cheb;
  s->legendre = inner->legendre;
  s->real_phys = inner->real_phys;
  s->real_spec = inner->real_spec;
  s->nphys = inner->nphys;
  s->nspec = inner->nspec;
  s->phys_bytes = inner->phys_bytes;
  s->spec_bytes = inner->spec_bytes;
  s->inner = inner;
  for (int c = 0; c < ndim; ++c) {
    const int d = order[c];
    s->perm[d] = c;
    s->kinds[d] = ck[c];
    s->n[d] = cn[c];
    s->spec[d] = inner->spec[c];
    s->dom[2 * d] = inner->dom[2 * c];
    s->dom[2 * d + 1] = inner->dom[2 * c + 1];
  }
  const size_t wb = std::max(s->phys_bytes, s->spec_bytes);
  cudaError_t e = cudaMalloc(&s->P1, wb);
  if (e == cudaSuccess) e = cudaMalloc(&s->P2, wb);
  if (e != cudaSuccess) {
    cudaFree(s->P1);
    cudaFree(s->P2);
    sgm_space_destroy(inner);
    delete s;
    return set_error(SGM_ERR_ALLOC, "workspace: %s", cudaGetErrorString(e));
  }
  *out = s;
  return SGM_OK;
}

// array layout of s (which = SGM_PHYSICAL / SGM_SPECTRAL) -> canonical layout, and back
int to_canonical(const sgm_space* s, int which, const void* in, void* out, cudaStream_t st) {
  const bool phys = which == SGM_PHYSICAL;
  const int64_t* shape = phys ? s->n : s->spec;
  const size_t elem = (phys ? s->real_phys : s->real_spec) ? s->relem() : s->celem();
  return permute(in, out, s->ndim, shape, s->perm, elem, st);
}

int from_canonical(const sgm_space* s, int which, const void* in, void* out, cudaStream_t st) {
  const bool phys = which == SGM_PHYSICAL;
  const size_t elem = (phys ? s->real_phys : s->real_spec) ? s->relem() : s->celem();
  int64_t cshape[3];
  int back[3];
  for (int d = 0; d < s->ndim; ++d) {
    cshape[s->perm[d]] = phys ? s->n[d] : s->spec[d];
    back[s->perm[d]] = d;
  }
  return permute(in, out, s->ndim, cshape, back, elem, st);
}

}  // namespace sgm
