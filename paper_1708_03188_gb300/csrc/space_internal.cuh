// space_internal.cuh - the sgm_space object shared by the host translation units
// (space.cu, gl.cu).
#pragma once
#include <cuda.h>
#include <map>
#include <stdint.h>

#include "../../include/sgm.h"
#include "common.cuh"

struct sgm_space {
  static constexpr uint32_t kMagic = 0x5347'4d53u;
  uint32_t magic = kMagic;
  int device = 0;
  int ndim = 0;
  int kinds[3] = {0, 0, 0};
  int64_t n[3] = {1, 1, 1};
  double dom[6] = {0, 0, 0, 0, 0, 0};
  int prec = SGM_F64;
  bool cheb = false;       // axis 0 is a polynomial axis (Chebyshev or Legendre family)
  bool legendre = false;   // axis 0 is a Legendre basis (legendre.cu)
  bool real_phys = false;  // physical array is real
  bool real_spec = false;  // spectral array is real (1-D Chebyshev)
  int64_t spec[3] = {1, 1, 1};
  long nphys = 0, nspec = 0;
  size_t phys_bytes = 0, spec_bytes = 0;
  std::map<int, void*> tw;   // length -> exp(-2 pi i k / L)
  std::map<int, void*> twf;  // length -> pass twiddle tables of the compile-time FFT engine
  void* dctw = nullptr;      // exp(-i pi k / (2N))
  double* tab = nullptr;     // Galerkin coefficient tables (Dirichlet or biharmonic)
  void* W1 = nullptr;
  void* W2 = nullptr;
  double* scratch = nullptr;
  long scratch_threads = 0;
  int2* groups = nullptr;    // (a, b) table of the four-column grouping of the self-contained eliminations
  long ngroups = 0;
  int solve_nc = 1;          // columns per elimination thread (1, 2 or 4)
  // factorisation tables of the 3-D Dirichlet and biharmonic eliminations (k_solve.cu
  // launch_factor, one entry per pair of columns +-l1 and parity): two slots of rows x values x
  // fact_threads doubles, each keyed by the operator and column layout it holds (basis, a, b, c,
  // n2) and replaced least recently used; the scratch holds the factored solves' rows (one thread
  // per column and parity) for fact_scratch_threads threads
  double* fact[2] = {nullptr, nullptr};
  double fact_key[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
  bool fact_valid[2] = {false, false};
  unsigned long fact_use[2] = {0, 0};
  unsigned long fact_clock = 0;
  long fact_threads = 0;          // table threads of a slot
  long fact_scratch_threads = 0;  // threads of a factored solve (scratch rows)
  int cheb_tc = 0;           // 1: Chebyshev axis by the tensor-core contraction (k_cheb_tc.cu)
  void* tc_img[3] = {nullptr, nullptr, nullptr};  // contraction matrices per ChebMode
  void* pdx_tab = nullptr;   // Shen-to-Chebyshev stencil coefficients of sgm_project_dx (project.cu)
  void* leg_mat[3] = {nullptr, nullptr, nullptr};  // Legendre axis-0 matrices per ChebMode (legendre.cu)
  double* leg_band = nullptr;   // band entries of the Legendre Galerkin matrices, 6 per basis row
  double* leg_scratch = nullptr;
  long leg_threads = 0;
  // streaming pipeline of the physical-to-physical solves on FP32 spaces (k_stream.cu): W1 and W2
  // (both complex64) hold the intermediates with the last axis padded to hp (even)
  // coefficients per row, so every row starts on a 16-byte boundary; TMA tensor maps over W1 for
  // the Chebyshev passes (as floats, 2-D) and the strided passes (3-D)
  // a space whose axes are not in the canonical order (axes.cu) is a view of the canonical space
  // `inner`: perm[d] = canonical axis of array axis d; P1, P2 = canonical-layout workspaces
  sgm_space* inner = nullptr;
  int perm[3] = {0, 1, 2};
  void* P1 = nullptr;
  void* P2 = nullptr;
  bool stream = false;
  // sgm_space_solve_events: events recorded around the elimination of the physical-to-physical solves
  cudaEvent_t ev_solve_begin = nullptr, ev_solve_end = nullptr;
  int hp = 0;
  long inner_p = 0;          // padded column count of the intermediates (M1 hp, or hp)
  CUtensorMap map_w1, map_w1s;

  size_t celem() const { return prec == SGM_F32 ? 8 : 16; }
  size_t relem() const { return prec == SGM_F32 ? 4 : 8; }
};

namespace sgm {
// pass tables of the compile-time FFT engine for length L on this space's device and
// precision (nullptr if L has no compiled kernel); owned by the space
int need_twf(sgm_space* s, int L, const void** out);
int space_check(const sgm_space* s);
// spaces in another axis order (axes.cu): whether kinds are in the canonical order (polynomial
// axis first, R2C axis last), the creation of a permuted view, and the layout permutations
bool canonical_axes(int ndim, const int* kinds);
int permuted_create(sgm_space** out, int ndim, const int* kinds, const int64_t* n, const double* domain, int precision);
int to_canonical(const sgm_space* s, int which, const void* in, void* out, cudaStream_t st);
int from_canonical(const sgm_space* s, int which, const void* in, void* out, cudaStream_t st);
// mass solve B u = data in place on FP64 spectral data of a space whose axis 0 is a Shen basis
// (space.cu; uses the space's elimination scratch)
int space_mass_solve_f64(sgm_space* s, void* data, cudaStream_t st);
// device table of the compile-time FFT engine for length L (caller frees)
int make_fast_twiddles(int precision, int L, void** out);
// stencil coefficient table of sgm_project_dx for a space with a Chebyshev axis (project.cu);
// stored in s->pdx_tab, freed with the space
int build_project_table(sgm_space* s);
// Legendre axis 0 (legendre.cu): tables, matrices and solve scratch of a new space, plus the
// tensor-core images of its matrices in s->tc_img when tc_images (FP32, N <= 128; all freed with
// the space); one axis-0 pass (mode: ChebMode; wide: the spectral side is FP64 on an FP32 space);
// the banded FP64 solve of a (S - 2 k2 A + k2^2 B) + b (A - k2 B) + c B, the biharmonic weak form
// (a Dirichlet problem a lap(u) + b u = f is (0, a, b): its tables have S = 0), on spectral data
// of type TS (float or double)
int legendre_build(sgm_space* s, bool tc_images);
// streaming passes (k_stream.cu): lengths with a kernel, the launches (Chebyshev mode
// kChebScalar: map over the complex64 intermediate, complex64 spectral out; kChebBackward: map over
// the complex64 spectral solution, transformed in place) and the tensor-map encoder (tma.cuh)
bool cheb_stream_length(int N);
cudaError_t launch_cheb_stream(int mode, int N, const CUtensorMap& map, void* out, long inner, int basis,
                               const float2* twf, const float2* dctw, cudaStream_t s);
bool rows_stream_length(int LF);
bool strided_stream_length(int L);
cudaError_t launch_rows_stream(int mode, int LF, const void* in, void* out, long nrows, int hp, const float2* twf,
                               const float2* tw_L, cudaStream_t s);
cudaError_t launch_strided_stream(bool inverse, int L, const CUtensorMap& map, float2* data, long outer, int hp,
                                  const float2* twf, cudaStream_t s);
cudaError_t encode_tiled_map(CUtensorMap* map, CUtensorMapDataType dtype, int rank, const void* base,
                             const uint64_t* dims, const uint64_t* strides, const uint32_t* box);
int legendre_pass(sgm_space* s, int mode, const void* in, void* out, cudaStream_t st, bool wide);
template <typename TS>
int legendre_solve(sgm_space* s, double a, double b, double c, const void* in, void* out, const Wavenumbers& wn,
                   cudaStream_t st);
}  // namespace sgm
