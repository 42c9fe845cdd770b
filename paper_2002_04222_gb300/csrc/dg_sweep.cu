// The fused BRJ sweep (Eq. precond-Jacobi, sweeps j >= 2): one kernel per
// sweep that forms y_e = q_e - (L+U)_e q^(j-1) of an element in shared memory
// and multiplies it by the element's inverse block in the same block of
// threads.  Kept in its own translation unit so that it compiles in parallel
// with the build kernels.
#include <type_traits>
#include "dg_brj_apply.cuh"
#include "dg_precond.h"

namespace dg {

// columns of each chunk of the block prefetched to L2 at the start of a sweep
constexpr int SWEEP_PREFETCH_COLS = 16;

// One whole relaxation sweep per element (Eq. precond-Jacobi, j >= 2):
// y_e = q_e - (L+U)_e qprev is formed in shared memory by the off-diagonal
// product and multiplied by the block in the same block of threads, so y never
// goes through HBM and the neighbour gather overlaps other blocks' streams.
// Launched with exactly the bound's thread count; qprev and out must differ.
template <int DIM, int P, int Q, typename TB, typename TJ, bool CV>
__global__ void DG_DIAG_BOUNDS(TB)
    brj_sweep_kernel(const __grid_constant__ Tables tab, const ElemGeo* __restrict__ geo,
                     const double* __restrict__ minv, const TJ* __restrict__ Jo,
                     const int32_t* __restrict__ nbr, const double* __restrict__ qprev,
                     const double* __restrict__ q, double dta, const TB* __restrict__ blocks,
                     int nb, int ld, int split, double omega, double* __restrict__ out) {
  using TA = typename Vec16<TB>::TA;
  constexpr int NTH = sizeof(TB) == 2 ? 512 : 256;
  extern __shared__ unsigned char smraw[];
  TA* sy = reinterpret_cast<TA*>(smraw);                 // [nb]
  TA* part = sy + nb;                                    // [split][ld]
  const int e = blockIdx.x;
  // the block's first columns of each thread group's chunk start their way
  // from DRAM while the off-diagonal gather runs (a bounded share of the
  // block, so that the prefetches of the resident blocks fit in L2)
  if (threadIdx.x >= 32 && threadIdx.x < 32 + split) {
    const int chunk = (nb + split - 1) / split;
    const int c0 = (threadIdx.x - 32) * chunk;
    const int nc = min(SWEEP_PREFETCH_COLS, min(chunk, nb - c0));
    if (nc > 0)
      prefetch_l2(blocks + (long long)e * nb * ld + (long long)c0 * ld, sizeof(TB) * (size_t)nc * ld);
  }
  offdiag_element<DIM, P, Q, TA, TJ, CV, NTH>(tab, geo, minv, Jo, nbr, qprev, q, dta, e,
                                              [&](int i, double v) { sy[i] = (TA)v; });
  __syncthreads();
  diag_element<TB>(blocks, nb, ld, split, sy, part, qprev, omega, out, e);
}

template <int D, int P, int Q, typename TB, bool CV>
static dg_status sweep_launch(dg_precond_s* pc, const double* qprev, const double* q, double* out,
                              cudaStream_t s) {
  using V = Vec16<TB>;
  using TJ = typename std::conditional<std::is_same<TB, double>::value, double, float>::type;
  constexpr int NTH = sizeof(TB) == 2 ? 512 : 256;  // the kernel's bound and its block size
  dg_mesh_s* m = pc->mesh;
  const int nb = pc->nb, ld = round_up8(nb);
  const int nrq = ld / V::W;
  int split = NTH / nrq;
  if (split < 1) split = 1;
  if (nrq * split > NTH) return DG_ERR_UNSUPPORTED;
  const size_t sm = sizeof(typename V::TA) * ((size_t)nb + (size_t)split * ld);
  DG_PROF(K_BRJ_SWEEP, s, brj_sweep_kernel<D, P, Q, TB, TJ, CV><<<m->E, NTH, sm, s>>>(
      m->tab, m->geo, m->minv, (const TJ*)pc->jo, pc->nbr, qprev, q, pc->dt_a,
      (const TB*)pc->blocks, nb, ld, split, pc->omega, out));
  DG_LAUNCHED(1);
  return DG_OK;
}

template <int D, int P, int Q, typename TB>
static dg_status sweep_dispatch(dg_precond_s* pc, const double* qprev, const double* q,
                                double* out, cudaStream_t s) {
  if (!pc->mesh->curved) return sweep_launch<D, P, Q, TB, false>(pc, qprev, q, out, s);
  if constexpr (has_curved<D, P, Q>()) return sweep_launch<D, P, Q, TB, true>(pc, qprev, q, out, s);
  return DG_ERR_UNSUPPORTED;
}

dg_status dispatch_sweep(dg_precond_s* pc, const double* qprev, const double* q, double* out,
                                cudaStream_t s) {
  dg_mesh_s* m = pc->mesh;
#define DG_S(D_, P_, Q_)                                                          \
  if (m->dim == D_ && m->P == P_ && m->Q == Q_) {                                 \
    if (pc->precision == DG_PREC_FP64)                                            \
      return sweep_dispatch<D_, P_, Q_, double>(pc, qprev, q, out, s);            \
    if (pc->precision == DG_PREC_FP32)                                            \
      return sweep_dispatch<D_, P_, Q_, float>(pc, qprev, q, out, s);             \
    return sweep_dispatch<D_, P_, Q_, __nv_bfloat16>(pc, qprev, q, out, s);       \
  }
  DG_PREC_INSTANCES(DG_S)
#undef DG_S
  return DG_ERR_UNSUPPORTED;
}

}  // namespace dg
