// gpe_tma.cuh -- persistent Crank-Nicolson line sweeps whose tiles move by
// TMA (the tensor-memory accelerator of sm_90 and later): the y/z sweeps
// (a3, a4 of the split step; "Solution method" of the paper) of FP32 states
// on grids whose lines are too large to stay in L2.
//
// One CTA per SM (or two, where their stages fit) walks tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...; a tile is 32 neighbouring lines (32 consecutive
// x positions) times the whole line, laid out in shared memory as [point k]
// [line], 256 bytes per point -- the same lane = line, warp = segment mapping
// as colsweep_body, read conflict-free.  Three stages: while tile t is solved
// in place in its stage, tile t + 1 has landed or is landing in the next, and
// the stage of tile t - 1 is being written back by a TMA store and then
// refilled with tile t + 2.  A single thread issues one bulk-tensor load and
// one bulk-tensor store per tile, so no thread spends instructions on
// per-element addresses, predicates or copies; the solve is the segment scan
// of gpe_sweep2.cuh (the same increment-form recurrences, carried at half
// scale, with the exact segment carries), without per-point bounds tests on
// the segments that lie wholly inside the line.
//
// The two end points of every line are held at zero (R5): they are cleared in
// the staged tile before the solve, so the solve reads them as zeros and the
// store writes zeros there.  Lines past the grid's last x position (a partial
// tile) are loaded as zeros by the TMA unit and clipped by its store.
//
// Every wait on a stage's mbarrier is bounded by the global timer: past the
// limit the CTA records GPE_TMA_ERR_TIMEOUT in the handle's device error flag
// (the host returns GP_ERR_TIMEOUT at its next synchronising call), waits --
// again bounded -- for its other loads in flight, and returns.
#pragma once
#include <cuda.h>

#include "gpe_sweep2.cuh"

namespace gpe {

constexpr int kTmaStages = 3;
constexpr int GPE_TMA_ERR_TIMEOUT = 1;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity of the mbarrier to complete, for
// at most limit_ns nanoseconds of global time; false if the limit passed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}

// TMA tile load of the box at (c0, c1, c2) into shared memory, completing
// its bytes on the mbarrier.
__device__ __forceinline__ void tma_load3(const CUtensorMap* map, unsigned dst, unsigned bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// TMA tile store of shared memory to the box at (c0, c1, c2).
__device__ __forceinline__ void tma_store3(const CUtensorMap* map, unsigned src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<unsigned long long>(map)),
               "r"(src), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory made visible to the TMA unit
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(map)) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Barrier 1 over the consumer warps only (the producer warp never joins it).
__device__ __forceinline__ void consumers_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
__device__ __forceinline__ bool consumers_or(int nthreads, bool v) {
  unsigned r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)v), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Arguments beyond the sweep's own: the tile grid of the sweep and the
// handle's error flag.
struct TmaTiles {
  int nxt;        // tiles across x (ceil(nx / 32))
  int ntiles;     // nxt * (number of lines' other transverse positions)
  unsigned long long limit_ns;  // bound of every mbarrier wait
  int expect_extra;  // bytes added to every expected transaction count (0; a test sets it to make a wait run out)
  int* err;          // device error flag (GPE_TMA_ERR_*), 0 = fine
  int depth;         // x sweep: segments whose carries reach a segment (the others' tables are below 2^-48)
};

// Forward pass of the segment of this thread from the staged tile (rows 0
// and n - 1 already zero); FULL: the segment lies wholly inside 1..M.
template <bool IMAG, int SEG, bool FULL>
__device__ __forceinline__ void tma_forward(const float2* buf, int lane, const float2* al, int k0, int M,
                                            float2 (&e)[SEG]) {
  // rows 0..M+1 of the tile (a failed check reads zero)
  auto row = [&](int k) {
    return GPE_CHECK(k >= 0 && k <= M + 1, 281) ? buf[k * 32 + lane] : make_float2(0.f, 0.f);
  };
  float2 pm = row(k0 - 1), pc = row(k0);
  float2 prev = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int k = k0 + j;
    float2 pn;
    if (FULL) pn = row(k + 1);
    else pn = (k + 1 <= M + 1) ? row(k + 1) : make_float2(0.f, 0.f);
    const float2 t = make_float2(prev.x + neg_lap(pm.x, pn.x, pc.x), prev.y + neg_lap(pm.y, pn.y, pc.y));
    float2 v = make_float2(0.f, 0.f);
    if (FULL || k <= M) v = cf_mul<float, IMAG>(al[k], t);
    e[j] = v;
    prev = v;
    pm = pc;
    pc = pn;
  }
}

// The segment carries of seg_carries (gpe_sweep2.cuh) with the per-point
// bounds tests dropped on full segments.
// k0: the segment's first point; M: the last point of the recurrences (points
// beyond it, FULL = false only, are zero).
// The consumer warps (32 nseg threads) synchronise on barrier 1.
template <bool IMAG, int SEG, bool FULL>
__device__ __forceinline__ void tma_carries(float2 (&z)[SEG], const float2* sc, int n, float2 (*cf)[33],
                                            float2 (*cb)[33], int s, int nseg, int lane, int k0, int M,
                                            int cdepth, int cpts) {
  const int dep = cdepth > 0 ? cdepth : 16;
  const bool whole = FULL || k0 + SEG - 1 <= M;  // (cpts: 4, 8, 12 or 0 = every point, as in seg_carries)
  const float2* al = sc;
  const float2* gf = sc + n;
  const float2* gb = sc + 2 * n;
  const float2* Pf = sc + 3 * n;
  const float2* Pb = Pf + 256;
  {
    float2 Bend = z[SEG - 1];
    if (!FULL) {
#pragma unroll
      for (int j = 0; j < SEG; ++j)
        if (k0 + j == M) Bend = z[j];
    }
    cf[s][lane] = Bend;
  }
  consumers_sync(32 * nseg);
  float2 Ein = make_float2(0.f, 0.f);
  for (int q = max(0, s - dep); q < s; ++q) Ein = cf_fma<float, IMAG>(Pf[q * 16 + s - 1], cf[q][lane], Ein);
  auto fwd = [&](auto nj) {
#pragma unroll
    for (int j = 0; j < decltype(nj)::value; ++j) {
      const int k = k0 + j;
      if (FULL || k <= M) z[j] = cf_fma<float, IMAG>(gf[k], Ein, z[j]);
    }
  };
  if (SEG > 4 && cpts == 4) fwd(std::integral_constant<int, (SEG > 4 ? 4 : SEG)>());
  else if (SEG > 8 && cpts == 8) fwd(std::integral_constant<int, (SEG > 8 ? 8 : SEG)>());
  else if (SEG > 12 && cpts == 12) fwd(std::integral_constant<int, (SEG > 12 ? 12 : SEG)>());
  else fwd(std::integral_constant<int, SEG>());
  float2 next = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = SEG - 1; j >= 0; --j) {
    const int k = k0 + j;
    if (FULL || k <= M) next = cf_fma<float, IMAG>(al[k], next, z[j]);
    else next = make_float2(0.f, 0.f);
    z[j] = next;
  }
  cb[s][lane] = z[0];
  consumers_sync(32 * nseg);
  float2 Zin = make_float2(0.f, 0.f);
  const int qe = min(nseg, s + 1 + dep);
  for (int q = s + 1; q < qe; ++q) Zin = cf_fma<float, IMAG>(Pb[q * 16 + s + 1], cb[q][lane], Zin);
  auto bwd = [&](auto nj) {
#pragma unroll
    for (int j = SEG - decltype(nj)::value; j < SEG; ++j) {
      const int k = k0 + j;
      if (FULL || k <= M) z[j] = cf_fma<float, IMAG>(gb[k], Zin, z[j]);
    }
  };
  if (SEG > 4 && whole && cpts == 4) bwd(std::integral_constant<int, (SEG > 4 ? 4 : SEG)>());
  else if (SEG > 8 && whole && cpts == 8) bwd(std::integral_constant<int, (SEG > 8 ? 8 : SEG)>());
  else if (SEG > 12 && whole && cpts == 12) bwd(std::integral_constant<int, (SEG > 12 ? 12 : SEG)>());
  else bwd(std::integral_constant<int, SEG>());
}

// The carries of the even-aligned x sweep (every segment full), truncated to
// what FP32 can see: the carry into a segment is taken from the `depth`
// segments before (after) it only, and applied to its first (last) NJ points
// only.  The host picks depth and NJ so that every table entry left out --
// the products of the recurrence coefficients over the points and segments a
// carry crosses -- is at most 2^-48 in magnitude: an omitted term is below
// 2^-48 of the carried value, 2^-24 of an FP32 rounding of it.  With
// |alpha| ~ 0.01 (the 256^3 quench) a carry dies within 8 points of a
// segment's end and never crosses a whole segment.
template <bool IMAG, int SEG, int NJ>
__device__ __forceinline__ void tma_carries_x(float2 (&z)[SEG], const float2* sc, int n, float2 (*cf)[33],
                                              float2 (*cb)[33], int s, int nseg, int lane, int k0, int depth) {
  static_assert(NJ >= 1 && NJ <= SEG, "points that take a carry");
  const float2* al = sc;
  const float2* gf = sc + n;
  const float2* gb = sc + 2 * n;
  const float2* Pf = sc + 3 * n;
  const float2* Pb = Pf + 256;
  // (k0 and NJ are even and the tables start on 16-byte boundaries: the
  // coefficients of two points come in one 16-byte load)
  auto pair = [](const float2* t, int k) { return *reinterpret_cast<const float4*>(t + k); };
  cf[s][lane] = z[SEG - 1];
  consumers_sync(32 * nseg);
  float2 Ein = make_float2(0.f, 0.f);
  for (int q = max(0, s - depth); q < s; ++q) Ein = cf_fma<float, IMAG>(Pf[q * 16 + s - 1], cf[q][lane], Ein);
#pragma unroll
  for (int j = 0; j < NJ; j += 2) {
    const float4 g2 = pair(gf, k0 + j);
    z[j] = cf_fma<float, IMAG>(make_float2(g2.x, g2.y), Ein, z[j]);
    z[j + 1] = cf_fma<float, IMAG>(make_float2(g2.z, g2.w), Ein, z[j + 1]);
  }
  float2 next = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = SEG - 2; j >= 0; j -= 2) {
    const float4 a2 = pair(al, k0 + j);
    next = cf_fma<float, IMAG>(make_float2(a2.z, a2.w), next, z[j + 1]);
    z[j + 1] = next;
    next = cf_fma<float, IMAG>(make_float2(a2.x, a2.y), next, z[j]);
    z[j] = next;
  }
  cb[s][lane] = z[0];
  consumers_sync(32 * nseg);
  float2 Zin = make_float2(0.f, 0.f);
  const int qe = min(nseg, s + 1 + depth);
  for (int q = s + 1; q < qe; ++q) Zin = cf_fma<float, IMAG>(Pb[q * 16 + s + 1], cb[q][lane], Zin);
#pragma unroll
  for (int j = SEG - NJ; j < SEG; j += 2) {
    const float4 g2 = pair(gb, k0 + j);
    z[j] = cf_fma<float, IMAG>(make_float2(g2.x, g2.y), Zin, z[j]);
    z[j + 1] = cf_fma<float, IMAG>(make_float2(g2.z, g2.w), Zin, z[j + 1]);
  }
}

// Solve of one staged tile in place (every thread of the block); returns this
// thread's Simpson-weighted norm contribution (LAST).  c = the lines' other
// transverse index (z for y lines, y for z lines), i = the line's x index.
template <bool IMAG, bool LAST, int SEG, bool CLOSE, bool FULL>
__device__ __forceinline__ float tma_solve_tile(const Sweep2Args<float>& A, float2* buf, const float2* sc,
                                                float2 (*cf)[33], float2 (*cb)[33], int i, int c, int nseg) {
  const LineGeom& G = A.geom;
  const int n = G.n, M = n - 2;
  const int lane = threadIdx.x & 31, s = threadIdx.x >> 5;
  const int k0 = 1 + s * SEG;
  float2 z[SEG];
  tma_forward<IMAG, SEG, FULL>(buf, lane, sc, k0, M, z);
  tma_carries<IMAG, SEG, FULL>(z, sc, n, cf, cb, s, nseg, lane, k0, M, A.cdepth, A.cpts);
  float tacc = 0.f;
  const long st = G.stride;
  const long qb = G.axis == 1 ? (long)i + (long)G.nx * G.ny * c : (long)i + (long)G.nx * c;
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int k = k0 + j;
    if (FULL || k <= M) {
      float2 u = sub2<float>(buf[k * 32 + lane], z[j]);
      if constexpr (CLOSE) {
        const int jy = G.axis == 2 ? c : k, kz = G.axis == 2 ? k : c;
        u = half_phase<float, IMAG>(A, u, qb + (long)k * st, i, jy, kz);
      }
      buf[k * 32 + lane] = u;
      if (LAST) tacc = fmaf(A.w_axis[k], u.x * u.x + u.y * u.y, tacc);
    }
  }
  return tacc;
}

// The producer of a persistent TMA sweep: one thread (lane 0 of the last
// warp) walks this CTA's tiles; for tile number it it first stores the tile
// kTmaStages earlier, whose stage the consumer warps have finished (their
// arrivals on empty[stage]), waits until the store has read the stage, and
// refills the stage with tile it (its bytes completing on full[stage]); then
// the tiles still unstored.  Loads thus run kTmaStages tiles ahead of the
// consumers and no consumer ever waits for a store.  Every wait is bounded:
// on a timeout, or when the consumers gave up (*abort), the producer stops
// issuing, waits -- bounded -- for the loads it issued, and for its stores.
template <typename LoadF, typename StoreF>
__device__ __forceinline__ void tma_producer(const TmaTiles& T, unsigned full0, unsigned empty0,
                                             volatile int* abort, LoadF load, StoreF store) {
  int it = 0;
  bool stop = false;
  for (int t = blockIdx.x; t < T.ntiles; t += gridDim.x, ++it) {
    const int st = it % kTmaStages;
    if (it >= kTmaStages) {
      if (!mbar_wait_bounded(empty0 + 8u * st, (unsigned)(it / kTmaStages - 1) & 1u, T.limit_ns) || *abort) {
        stop = true;
        break;
      }
      store(t - kTmaStages * (int)gridDim.x, st);
      bulk_commit();
      bulk_wait_read<0>();
    }
    load(t, st);
  }
  if (!stop) {
    for (int q = it > kTmaStages ? it - kTmaStages : 0; q < it; ++q) {
      const int st = q % kTmaStages;
      if (!mbar_wait_bounded(empty0 + 8u * st, (unsigned)(q / kTmaStages) & 1u, T.limit_ns) || *abort) {
        stop = true;
        break;
      }
      store(blockIdx.x + q * (int)gridDim.x, st);
      bulk_commit();
    }
  }
  if (stop) {
    atomicExch(T.err, GPE_TMA_ERR_TIMEOUT);
    // the loads issued (the last one into each stage) have landed before the CTA ends
    for (int q = it - 1; q >= 0 && q >= it - kTmaStages; --q)
      mbar_wait_bounded(full0 + 8u * (q % kTmaStages), (unsigned)(q / kTmaStages) & 1u, T.limit_ns);
  }
  bulk_wait_all();  // the stores have completed before the grid does
}

// The persistent TMA-pipelined y/z sweep (FP32 state).  tm: the state as a
// 3d tensor of 8-byte elements (nx, ny, nz) with the box (32, n, 1) for y
// lines or (32, 1, n) for z lines.  blockDim.x = 32 (nseg + 1): nseg <= 16
// consumer warps (warp = segment) and one producer warp; dynamic shared
// memory: the coefficients (3n + 512 complex), then, from the next 1024-byte
// boundary, kTmaStages tiles of 32 n complex values.
template <bool IMAG, bool LAST, int SEG, bool CLOSE>
__global__ void __launch_bounds__(544, 1) tmacol_kernel(const __grid_constant__ CUtensorMap tm, Sweep2Args<float> A,
                                                        TmaTiles T) {
  extern __shared__ __align__(1024) unsigned char tma_smem_raw[];
  __shared__ __align__(8) unsigned long long full[kTmaStages], empty[kTmaStages];
  __shared__ float2 cf[16][33], cb[16][33];
  __shared__ int abort_flag;
  const LineGeom& G = A.geom;
  const int n = G.n, M = n - 2;
  const int lane = threadIdx.x & 31, s = threadIdx.x >> 5, nseg = (blockDim.x >> 5) - 1;
  float2* sc = reinterpret_cast<float2*>(tma_smem_raw);
  const unsigned base = smem_u32(tma_smem_raw);
  const unsigned coef_bytes = (unsigned)(3 * n + 512) * 8u;
  const unsigned tiles0 = (base + coef_bytes + 1023u) & ~1023u;  // first stage, 1024-byte aligned
  const unsigned tile_bytes = 32u * (unsigned)n * 8u;
  float2* tiles = reinterpret_cast<float2*>(tma_smem_raw + (tiles0 - base));
  const bool yaxis = G.axis == 1;
  auto coords = [&](int t, int& c0, int& c1, int& c2) {
    const int ix = t % T.nxt, oc = t / T.nxt;
    c0 = ix * 32;
    c1 = yaxis ? 0 : oc;
    c2 = yaxis ? oc : 0;
  };
  const unsigned full0 = smem_u32(&full[0]), empty0 = smem_u32(&empty[0]);
  if (threadIdx.x == 0) {
    prefetch_tmap(&tm);
    for (int st = 0; st < kTmaStages; ++st) {
      mbar_init(full0 + 8u * st, 1);
      mbar_init(empty0 + 8u * st, 32u * nseg);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  load_coefs<float>(A, sc, n);
  __syncthreads();  // barriers initialised, coefficients staged
  pdl_wait();       // the state is the previous kernel's output
  pdl_release();
  float tval = 0.f;
  if (s == nseg) {  // ---- producer warp
    if (lane == 0) {
      tma_producer(
          T, full0, empty0, &abort_flag,
          [&](int t, int st) {
            int c0, c1, c2;
            coords(t, c0, c1, c2);
            mbar_expect_tx(full0 + 8u * st, tile_bytes + (unsigned)T.expect_extra);
            tma_load3(&tm, tiles0 + (unsigned)st * tile_bytes, full0 + 8u * st, c0, c1, c2);
          },
          [&](int t, int st) {
            int c0, c1, c2;
            coords(t, c0, c1, c2);
            tma_store3(&tm, tiles0 + (unsigned)st * tile_bytes, c0, c1, c2);
          });
    }
    __syncwarp();
  } else {  // ---- consumer warps: warp = segment, lane = line
    const bool full_seg = 1 + (s + 1) * SEG - 1 <= M;  // this warp's segment lies inside the line
    int it = 0;
    for (int t = blockIdx.x; t < T.ntiles; t += gridDim.x, ++it) {
      const int st = it % kTmaStages;
      const bool ok = mbar_wait_bounded(full0 + 8u * st, (unsigned)(it / kTmaStages) & 1u, T.limit_ns);
      float2* buf = tiles + (size_t)st * 32 * n;
      if (ok && s == 0) {  // the end points are held at zero
        buf[lane] = make_float2(0.f, 0.f);
        buf[(n - 1) * 32 + lane] = make_float2(0.f, 0.f);
      }
      if (consumers_or(32 * nseg, !ok)) {
        if (threadIdx.x == 0) {
          abort_flag = 1;
          atomicExch(T.err, GPE_TMA_ERR_TIMEOUT);
        }
        break;
      }
      int c0, c1, c2;
      coords(t, c0, c1, c2);
      const int i = c0 + lane, c = yaxis ? c2 : c1;
      const float tacc = full_seg ? tma_solve_tile<IMAG, LAST, SEG, CLOSE, true>(A, buf, sc, cf, cb, i, c, nseg)
                                  : tma_solve_tile<IMAG, LAST, SEG, CLOSE, false>(A, buf, sc, cf, cb, i, c, nseg);
      if (LAST && i < G.nx) tval = fmaf(tacc, A.w_a[i] * A.w_b[c], tval);
      fence_async_smem();  // the solved tile is visible to the TMA unit ...
      mbar_arrive(empty0 + 8u * st);  // ... when the producer sees this stage done
    }
  }
  finish_norm<float, LAST>(tval, A.parts_out);
}

// ---------------------------------------------------------------- x sweep
// The x sweep with the sub-step N and the pending renormalisation factor
// (FIRST of a step; a1 + a2 of the split step) on the same three-stage TMA
// pipeline.  A tile is 32 x lines (consecutive lines L = j + ny k) times the
// whole line.  The tensor map views the state as (16, nx/16, nlines) 8-byte
// elements with the box (16, 1, 32) and the 128-byte swizzle, so one box is a
// 16-point chunk of 32 lines, 128 bytes per line, whose 16-byte units u
// (point pairs) sit at u ^ (line & 7); a tile is nx/16 such boxes, 4 KB
// each.  Lane = line, warp = segment: a warp reads one point pair of 32
// lines at a time with 16-byte loads, and the swizzle puts the 8 lines of
// every quarter warp in 8 different bank groups (no conflicts).
//
// Segments are aligned to even points: segment s covers points s SEG ..
// s SEG + SEG - 1 of the line, the end points included (the recurrences'
// coefficients are zero there, and the tables -- gf, gb and the carry tables
// -- are those of this segmentation), so with nx a multiple of 16 and SEG 8
// or 16 every segment is full and the solve has no bounds tests.  Each thread
// applies the pending factor and N to its own points in registers (no pass
// over the tile) and takes the point on either side of its segment, after N,
// from the neighbouring warps through two small shared arrays (one barrier).
// (Recomputing those two points instead, with no barrier, was 4 % slower.)
__device__ __forceinline__ unsigned swz_off(int l, int k) {
  // byte offset of point k of line l in a tile of 16-point chunks (k even: the pair k, k + 1)
  return (unsigned)(k >> 4) * 4096u + (unsigned)l * 128u + ((unsigned)(((k & 15) >> 1) ^ (l & 7)) << 4) +
         ((unsigned)(k & 1) << 3);
}

template <bool IMAG, int SEG, int NJ>
__global__ void __launch_bounds__(544, 1) tmarow_kernel(const __grid_constant__ CUtensorMap tm, Sweep2Args<float> A,
                                                        TmaTiles T) {
  static_assert(SEG == 8 || SEG == 16, "even-aligned segments of 8 or 16 points");
  extern __shared__ __align__(1024) unsigned char tma_smem_raw[];
  __shared__ __align__(8) unsigned long long full[kTmaStages], empty[kTmaStages];
  __shared__ float2 cf[16][33], cb[16][33];
  __shared__ float2 edge_l[16][32], edge_r[16][32];  // each segment's first and last point after N
  __shared__ float scl_smem;
  __shared__ int abort_flag;
  const LineGeom& G = A.geom;
  const int n = G.n;  // = nx, a multiple of 16
  const int lane = threadIdx.x & 31, s = threadIdx.x >> 5, nseg = (blockDim.x >> 5) - 1;
  float2* sc = reinterpret_cast<float2*>(tma_smem_raw);
  float* sv = reinterpret_cast<float*>(sc + 3 * n + 512);  // vx (harmonic potential along x)
  const unsigned base = smem_u32(tma_smem_raw);
  const unsigned coef_bytes = (unsigned)(3 * n + 512) * 8u + (unsigned)n * 4u;
  const unsigned tiles0 = (base + coef_bytes + 1023u) & ~1023u;
  const unsigned tile_bytes = 32u * (unsigned)n * 8u;
  const unsigned char* tiles_gen = tma_smem_raw + (tiles0 - base);
  const int nchunk = n >> 4;
  const unsigned full0 = smem_u32(&full[0]), empty0 = smem_u32(&empty[0]);
  if (threadIdx.x == 0) {
    prefetch_tmap(&tm);
    for (int st = 0; st < kTmaStages; ++st) {
      mbar_init(full0 + 8u * st, 1);
      mbar_init(empty0 + 8u * st, 32u * nseg);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  load_coefs<float>(A, sc, n);
  for (int k = threadIdx.x; k < n; k += blockDim.x) sv[k] = A.V ? 0.f : A.vx[k];
  pdl_wait();  // the state and the norm sums are the previous kernels' output
  pdl_release();
  if (s == 0) {
    const float f = A.parts_in ? (float)pending_factor_warp(A.parts_in, A.nparts_in, A.parts_wscale) : 1.f;
    if (lane == 0) scl_smem = f;
  }
  __syncthreads();  // barriers, coefficients, potential and factor ready
  if (s == nseg) {  // ---- producer warp
    if (lane == 0) {
      tma_producer(
          T, full0, empty0, &abort_flag,
          [&](int t, int st) {
            mbar_expect_tx(full0 + 8u * st, tile_bytes + (unsigned)T.expect_extra);
            const unsigned dst = tiles0 + (unsigned)st * tile_bytes;
            for (int b = 0; b < nchunk; ++b) tma_load3(&tm, dst + (unsigned)b * 4096u, full0 + 8u * st, 0, b, t * 32);
          },
          [&](int t, int st) {
            const unsigned src = tiles0 + (unsigned)st * tile_bytes;
            for (int b = 0; b < nchunk; ++b) tma_store3(&tm, src + (unsigned)b * 4096u, 0, b, t * 32);
          });
    }
    __syncwarp();
    return;
  }
  // ---- consumer warps: warp = segment, lane = line
  const float scl = scl_smem;
  const float inv_ny = 1.0f / (float)G.ny;
  // per-line part of N of this lane's line in tile t, vy[j] + vz[k] for the
  // line L = j + ny k: k from a float estimate of L / ny (exact to within one
  // for L < 2^24), corrected
  auto line_potential = [&](int t) -> float {
    const int L = t * 32 + lane;
    if (A.V || t >= T.ntiles || L >= G.nlines) return 0.f;
    int kq, jr;
    if (G.nlines < (1L << 24)) {
      kq = (int)((float)L * inv_ny);
      jr = L - kq * G.ny;
      if (jr < 0) {
        --kq;
        jr += G.ny;
      } else if (jr >= G.ny) {
        ++kq;
        jr -= G.ny;
      }
    } else {
      kq = L / G.ny;
      jr = L - kq * G.ny;
    }
    return A.vy[jr] + A.vz[kq];
  };
  float vnext = line_potential(blockIdx.x);
  const int k0 = s * SEG;
  int it = 0;
  for (int t = blockIdx.x; t < T.ntiles; t += gridDim.x, ++it) {
    const int st = it % kTmaStages;
    const bool ok = mbar_wait_bounded(full0 + 8u * st, (unsigned)(it / kTmaStages) & 1u, T.limit_ns);
    if (consumers_or(32 * nseg, !ok)) {  // all consumer warps take the same decision
      if (threadIdx.x == 0) {
        abort_flag = 1;
        atomicExch(T.err, GPE_TMA_ERR_TIMEOUT);
      }
      break;
    }
    const unsigned char* tb = tiles_gen + (size_t)st * tile_bytes;
    // a point pair of the staged tile (a failed check reads zeros, skips the store)
    auto ld2 = [&](int k) -> float4 {
      return GPE_CHECK(k >= 0 && k + 1 < n, 282) ? *reinterpret_cast<const float4*>(tb + swz_off(lane, k))
                                                 : make_float4(0, 0, 0, 0);
    };
    const int L = t * 32 + lane;
    const bool line_ok = L < G.nlines;
    // this tile's per-line potential (loaded one tile ahead), the next tile's issued now
    const float vline = vnext;
    vnext = line_potential(t + gridDim.x);
    // p[1..SEG]: the points of this segment; p[0], p[SEG + 1]: the points on
    // either side, after N, from the neighbouring segments' warps
    float2 p[SEG + 2];
#pragma unroll
    for (int j = 0; j < SEG; j += 2) {
      const float4 v = ld2(k0 + j);
      p[1 + j] = make_float2(v.x, v.y);
      p[2 + j] = make_float2(v.z, v.w);
    }
    const long gbase = (long)L * G.nx;
    // the potential at point j of p; with the harmonic trap the vx of four
    // points come in one 16-byte load
    auto vpt = [&](int j, const float4& v4) -> float {
      if (A.V) return line_ok ? A.V[gbase + k0 - 1 + j] : 0.f;
      const int q = (j - 1) & 3;
      return (q == 0 ? v4.x : q == 1 ? v4.y : q == 2 ? v4.z : v4.w) + vline;
    };
    auto v4at = [&](int j) -> float4 {  // vx of points k0 + (j - 1) .. + 3, j - 1 a multiple of 4
      return A.V ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(sv + k0 + j - 1);
    };
    if (IMAG) {
      float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 1; j <= SEG; ++j) {
        if (((j - 1) & 3) == 0) v4 = v4at(j);
        const float2 w = make_float2(p[j].x * scl, p[j].y * scl);  // the pending renormalisation
        p[j] = phase_direct<float, true>(w, vpt(j, v4), A.dt, A.g);
      }
    } else {
      // real time: every angle first; when all of the warp's are below 1/32
      // (1/8) one branch-free pass rotates them all with the short (long)
      // series of rot_coefs, else rot_neg per point
      float th[SEG + 1];
      bool small = true, tiny = true;
      float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 1; j <= SEG; ++j) {
        if (((j - 1) & 3) == 0) v4 = v4at(j);
        th[j] = phase_angle<float>(p[j], vpt(j, v4), A.dt, A.g);
        small = small && fabsf(th[j]) < 0.125f;
        tiny = tiny && fabsf(th[j]) < 0.03125f;
      }
      if (__all_sync(0xffffffffu, tiny)) {
#pragma unroll
        for (int j = 1; j <= SEG; ++j) {
          float sn, cm1;
          rot_coefs_series_short(th[j], sn, cm1);
          p[j] = rot_apply<float>(p[j], sn, cm1);
        }
      } else if (__all_sync(0xffffffffu, small)) {
#pragma unroll
        for (int j = 1; j <= SEG; ++j) {
          float sn, cm1;
          rot_coefs_series(th[j], sn, cm1);
          p[j] = rot_apply<float>(p[j], sn, cm1);
        }
      } else {
#pragma unroll
        for (int j = 1; j <= SEG; ++j) p[j] = rot_neg<float>(p[j], th[j]);
      }
    }
    if (s == 0) p[1] = make_float2(0.f, 0.f);  // the end points are held at zero
    if (s == nseg - 1) p[SEG] = make_float2(0.f, 0.f);
    // the segment's end points to the neighbours (every warp is past the
    // previous tile's reads of these arrays: the vote above is a barrier)
    edge_l[s][lane] = p[1];
    edge_r[s][lane] = p[SEG];
    consumers_sync(32 * nseg);
    p[0] = s > 0 ? edge_r[s - 1][lane] : make_float2(0.f, 0.f);
    p[SEG + 1] = s < nseg - 1 ? edge_l[s + 1][lane] : make_float2(0.f, 0.f);
    float2 z[SEG];
    {
      float2 prev = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        const float4 a2 = *reinterpret_cast<const float4*>(sc + k0 + (j & ~1));  // alpha of two points
        const float2 t2 = make_float2(prev.x + neg_lap(p[j].x, p[j + 2].x, p[j + 1].x),
                                      prev.y + neg_lap(p[j].y, p[j + 2].y, p[j + 1].y));
        prev = cf_mul<float, IMAG>((j & 1) ? make_float2(a2.z, a2.w) : make_float2(a2.x, a2.y), t2);
        z[j] = prev;
      }
    }
    tma_carries_x<IMAG, SEG, NJ>(z, sc, n, cf, cb, s, nseg, lane, k0, T.depth);
    unsigned char* tw = const_cast<unsigned char*>(tb);
#pragma unroll
    for (int j = 0; j < SEG; j += 2) {
      const float2 u0 = sub2<float>(p[1 + j], z[j]), u1 = sub2<float>(p[2 + j], z[j + 1]);
      if (GPE_CHECK(k0 + j + 1 < n, 283))
        *reinterpret_cast<float4*>(tw + swz_off(lane, k0 + j)) = make_float4(u0.x, u0.y, u1.x, u1.y);
    }
    fence_async_smem();
    mbar_arrive(empty0 + 8u * st);
  }
}

}  // namespace gpe
