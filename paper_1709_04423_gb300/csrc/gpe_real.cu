// gpe_real.cu -- a real imaginary-time state (gp_set_real_state, declared in
// include/gpe.h).
//
// In imaginary time the Crank-Nicolson coefficients (r = dt/(4 dx^2)) and the
// sub-step N (a real exponential) are real ("Solution method" of the paper),
// so a state with zero imaginary parts stays real and its imaginary parts are
// never read.  The handle then keeps np values of the state precision in
// rpsi (half the bytes of the complex state) and the sweeps take them
// directly (enqueue_sweep_real); the complex buffer psi serves as the staging
// copy that the observables, the reduced densities and gp_get_state read.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "gpe_common.cuh"
#include "gpe_internal.h"

namespace gpe {
namespace {

template <typename T>
__global__ void c2r_kernel(const c2_t<T>* __restrict__ psi, T* __restrict__ r, long np, int* __restrict__ nonreal) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (long)gridDim.x * blockDim.x) {
    const c2_t<T> v = psi[q];
    r[q] = v.x;
    if (v.y != T(0)) *nonreal = 1;  // any writer: the same value
  }
}

template <typename T>
__global__ void r2c_kernel(const T* __restrict__ r, c2_t<T>* __restrict__ psi, long np) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (long)gridDim.x * blockDim.x)
    psi[q] = mk<T>(r[q], T(0));
}

int grid_blocks(long np) { return (int)std::min<long>((np + 255) / 256, 152L * 8); }

}  // namespace

void materialize_complex(gp_handle* h) {
  if (!h->real_mode) return;
  if (h->prec == GP_F64)
    r2c_kernel<double><<<grid_blocks(h->np), 256, 0, h->work>>>((const double*)h->rpsi, (double2*)h->psi, h->np);
  else
    r2c_kernel<float><<<grid_blocks(h->np), 256, 0, h->work>>>((const float*)h->rpsi, (float2*)h->psi, h->np);
  count_launch();
}

int real_from_complex(gp_handle* h) {
  GP_CUDA(cudaMemsetAsync(h->real_flag, 0, sizeof(int), h->work));
  if (h->prec == GP_F64)
    c2r_kernel<double><<<grid_blocks(h->np), 256, 0, h->work>>>((const double2*)h->psi, (double*)h->rpsi, h->np,
                                                                h->real_flag);
  else
    c2r_kernel<float><<<grid_blocks(h->np), 256, 0, h->work>>>((const float2*)h->psi, (float*)h->rpsi, h->np,
                                                               h->real_flag);
  count_launch();
  int nonreal = 0;
  GP_CUDA(cudaMemcpyAsync(&nonreal, h->real_flag, sizeof(int), cudaMemcpyDeviceToHost, h->work));
  GP_CUDA(cudaStreamSynchronize(h->work));
  return nonreal ? fail(GP_ERR_STATE, "the state has nonzero imaginary parts: it cannot be held as a real state")
                 : GP_OK;
}

}  // namespace gpe

using namespace gpe;

extern "C" int gp_set_real_state(gp_handle* h, int real) {
  if (!h) return fail(GP_ERR_INVALID, "gp_set_real_state: NULL handle");
  if (real != 0 && real != 1) return fail(GP_ERR_INVALID, "gp_set_real_state: real must be 0 or 1");
  if ((real != 0) == h->real_mode) return GP_OK;
  if (real) {
    if (h->prec == GP_DF64) return fail(GP_ERR_INVALID, "gp_set_real_state: real states are FP32 or FP64");
    if (h->dim < 2 || h->geom != 0)
      return fail(GP_ERR_INVALID, "gp_set_real_state: real states are for 2d and 3d Cartesian grids");
    if (h->n[0] % 2) return fail(GP_ERR_INVALID, "gp_set_real_state: needs an even number of x points");
    // x lines take the shared-memory tile (two real lines per column): the
    // tile's segment shape if it was chosen, else its default one
    const int tseg = tile_seg(h->n[0] - 2);
    const bool tile_fits = (36L * h->n[0] + 512) * (long)h->esize <= 200L * 1024;
    if (h->seg_c == 0 || !tile_fits || (!h->tile_x && tseg == 0))
      return fail(GP_ERR_INVALID,
                  "gp_set_real_state: needs the x tile and segmented y/z sweeps (at most 514 points per axis, "
                  "and an x tile that fits in shared memory)");
    if (!h->tile_x) {
      h->tile_x = true;
      h->seg_x = tseg;
      h->pipe_x = false;
    }
    if (h->strang) return fail(GP_ERR_STATE, "gp_set_real_state: the Strang splitting takes the complex state");
  }
  int rc = join_in(h);
  if (rc) return rc;
  drop_graphs(h);
  if (real) {
    if (!h->rpsi && (rc = dev_alloc(h, &h->rpsi, (size_t)h->np * (h->prec == GP_F64 ? 8 : 4)))) return rc;
    if (!h->real_flag) {
      void* p = nullptr;
      if ((rc = dev_alloc(h, &p, 256))) return rc;
      h->real_flag = (int*)p;
    }
    if ((rc = real_from_complex(h))) return rc;
    h->real_mode = true;
  } else {
    materialize_complex(h);
    GP_CUDA(cudaGetLastError());
    h->real_mode = false;
  }
  return join_out(h);
}
