// gpe_reduce.cu -- reduced (integrated) densities: the density summed with
// the composite-Simpson weights over the axes that are dropped, on the grid of
// the axes that are kept (the paper's programs write reduced 1d and 2d
// densities; "Summary of revisions").  Declared in include/gpe.h.
//
// Two launches, deterministic: stage 1 runs one thread per (output point,
// chunk of the dropped index space) and accumulates w |phi|^2 in FP64 (|phi|^2
// itself in the state precision); stage 2 adds each output point's chunks in
// a fixed order (one thread per point, or one block per point when there are
// many chunks).  Output points are consecutive along the first kept axis, so
// with x kept a warp reads contiguous rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "gpe_common.cuh"
#include "gpe_internal.h"

namespace gpe {
namespace {

struct RedGeom {
  int nk, nd;                    // kept and dropped axes
  int kn[3], dn[3];              // their lengths (kept: x first; dropped: x first)
  long kst[3], dst[3];           // their point strides
  const double* dw[3];           // Simpson weights of the dropped axes (FP64)
  long nout, ndrop;
  int nchunks;
};

template <typename T>
__global__ void __launch_bounds__(256) reduce_stage1(const c2_t<T>* __restrict__ psi, RedGeom G,
                                                     double* __restrict__ parts) {
  const long o = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (o >= G.nout) return;
  long qb = 0, rem = o;
  for (int a = 0; a < G.nk; ++a) {
    qb += (rem % G.kn[a]) * G.kst[a];
    rem /= G.kn[a];
  }
  const long t0 = G.ndrop * c / G.nchunks, t1 = G.ndrop * (c + 1) / G.nchunks;
  // dropped coordinates of t0, then stepped with carries
  int cd[3] = {0, 0, 0};
  rem = t0;
  for (int a = 0; a < G.nd; ++a) {
    cd[a] = (int)(rem % G.dn[a]);
    rem /= G.dn[a];
  }
  double acc = 0.0;
  for (long t = t0; t < t1; ++t) {
    long q = qb;
    double w = 1.0;
    for (int a = 0; a < G.nd; ++a) {
      q += cd[a] * G.dst[a];
      w *= G.dw[a][cd[a]];
    }
    const c2_t<T> p = psi[q];
    const T dens = p.x * p.x + p.y * p.y;
    acc = fma(w, (double)dens, acc);
    for (int a = 0; a < G.nd; ++a) {  // next dropped point
      if (++cd[a] < G.dn[a]) break;
      cd[a] = 0;
    }
  }
  parts[(long)c * G.nout + o] = acc;
}

// few chunks: one thread per output point, chunks in order
__global__ void __launch_bounds__(256) reduce_stage2(const double* __restrict__ parts, RedGeom G,
                                                     double* __restrict__ out) {
  const long o = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= G.nout) return;
  double s = 0.0;
  for (int c = 0; c < G.nchunks; ++c) s += parts[(long)c * G.nout + o];
  out[o] = s;
}

// many chunks: one block per output point, a fixed-order block reduction
__global__ void __launch_bounds__(256) reduce_stage2_block(const double* __restrict__ parts, RedGeom G,
                                                           double* __restrict__ out) {
  __shared__ double smem[32];
  const long o = blockIdx.x;
  double v[1] = {0.0};
  for (int c = threadIdx.x; c < G.nchunks; c += blockDim.x) v[0] += parts[(long)c * G.nout + o];
  block_sum<1>(v, smem);
  if (threadIdx.x == 0) out[o] = v[0];
}

}  // namespace
}  // namespace gpe

using namespace gpe;

extern "C" int gp_reduced_density(gp_handle* h, int keep_mask, double* out, int out_on_device) {
  if (!h || !out) return fail(GP_ERR_INVALID, "gp_reduced_density: NULL argument");
  if (keep_mask < 1 || keep_mask >= (1 << h->dim))
    return fail(GP_ERR_INVALID, "gp_reduced_density: keep_mask must name at least one axis, and only axes < dim");
  RedGeom G = {};
  const long stride[3] = {1, (long)axis_len(h, 0), (long)axis_len(h, 0) * axis_len(h, 1)};
  G.nout = 1;
  G.ndrop = 1;
  for (int d = 0; d < h->dim; ++d) {
    if ((keep_mask >> d) & 1) {
      G.kn[G.nk] = h->n[d];
      G.kst[G.nk++] = stride[d];
      G.nout *= h->n[d];
    } else {
      G.dn[G.nd] = h->n[d];
      G.dst[G.nd] = stride[d];
      G.dw[G.nd++] = h->wd[d];
      G.ndrop *= h->n[d];
    }
  }
  // chunks of the dropped space so that about 128 K threads take part
  G.nchunks = (int)std::max<long>(1, std::min<long>({(131072 + G.nout - 1) / G.nout, G.ndrop, 4096L}));
  int rc = join_in(h);
  if (rc) return rc;
  const size_t need = (size_t)G.nchunks * G.nout + (out_on_device ? 0 : (size_t)G.nout);
  if (need > h->red_cap) {
    if (h->red_parts) {
      cudaStreamSynchronize(h->work);
      guarded_free(h->red_parts);
      for (auto& p : h->allocs)
        if (p == h->red_parts) p = nullptr;
      h->red_parts = nullptr;
      h->red_cap = 0;
    }
    void* p = nullptr;
    if ((rc = dev_alloc(h, &p, need * sizeof(double)))) return rc;
    h->red_parts = (double*)p;
    h->red_cap = need;
  }
  double* dout = out_on_device ? out : h->red_parts + (size_t)G.nchunks * G.nout;
  materialize_complex(h);  // a real state: its complex copy
  const void* psi = h->psi;
  if (h->prec == GP_DF64) {  // rounded to complex128 first
    df_to_c128(h, h->df_stage);
    psi = h->df_stage;
  }
  const dim3 grid1((unsigned)((G.nout + 255) / 256), (unsigned)G.nchunks);
  if (h->prec == GP_F32)
    reduce_stage1<float><<<grid1, 256, 0, h->work>>>((const float2*)psi, G, h->red_parts);
  else
    reduce_stage1<double><<<grid1, 256, 0, h->work>>>((const double2*)psi, G, h->red_parts);
  count_launch();
  if (G.nchunks > 64)
    reduce_stage2_block<<<(unsigned)G.nout, 256, 0, h->work>>>(h->red_parts, G, dout);
  else
    reduce_stage2<<<(unsigned)((G.nout + 255) / 256), 256, 0, h->work>>>(h->red_parts, G, dout);
  count_launch();
  GP_CUDA(cudaGetLastError());
  if (!out_on_device) {
    GP_CUDA(cudaMemcpyAsync(out, dout, (size_t)G.nout * sizeof(double), cudaMemcpyDeviceToHost, h->work));
    GP_CUDA(cudaStreamSynchronize(h->work));
  }
  return join_out(h);
}
