// Pipelined CTA tiles (launch modes 4 and 5), one launch per time step.
//
// The tile kernels of modes 0 and 1 run the three phases of a tile -- rows
// (properties, Eq. (ABC), interface and closure rows), line solves, stores --
// one after the other with block barriers between them, so while the block
// assembles rows the FP64 line solves wait and vice versa (in the mixed
// precision step the rows are FP32 work and the solves FP64 work).  Here the
// block's warps split into producers and consumers (a split chosen by the
// host and measured: three producers per consumer for the FP64 rows, which
// cost about twice the FP64 solves; 9 of 16 warps for the mixed step, whose
// FP32 rows cost about as much as its FP64 solves) with two row buffers:
// producers assemble tile k+1 into one buffer while consumers solve and store
// tile k from the other.  Buffers change hands through named barriers: a
// "full" barrier per buffer (producers arrive, consumers wait) and an "empty"
// barrier per buffer (consumers arrive, producers wait).  The axial fluxes
// handed from tile to tile stay with the producers.  A tile holds as many
// lines as the consumer warps solve at once.  The block's first tile, which
// the consumers would otherwise wait for with nothing to do, is assembled by
// all warps of the block together (one block barrier), so the pipeline fills
// in a fraction of the time of one tile; likewise the stores of its last
// tile, for which the producers would otherwise wait idle.  The mixed step
// moves every tile's stores to the producers (pipe_tiles_finish_by_producers).  The mixed-precision rows are
// kept as packed FP32 (a, c, d) per node -- the values the FP32 assembly
// produces, widened exactly by the consumers -- and the consumers hold the
// eliminated FP64 coefficients in registers, which leaves room in shared
// memory for more warps.
#include <cuda_runtime.h>

#include "ccell_fp64_task.cuh"
#include "ccell_mixed_task.cuh"

namespace ccell {

constexpr int kBarProd = 1, kBarCons = 2, kBarFull = 3, kBarEmpty = 5, kBarSolved = 5;

// Producer / consumer loops over the block's tiles; Buf(k) gives the row
// buffers of the k-th tile of the block, Produce / Consume run its phases.
template <bool ENERGY, bool TRACE, class Produce, class Solve, class Finish>
__device__ __forceinline__ void pipe_tiles(const StepArgs& a, EAcc& acc, Produce produce,
                                           Solve solve, Finish finish) {
  const int nw = blockDim.x >> 5, P = a.pipe_producers, C = nw - P, NT = blockDim.x;
  const bool producer = (int)(threadIdx.x >> 5) < P;
  const WarpGroup grp = producer ? WarpGroup{0, P, kBarProd} : WarpGroup{P, C, kBarCons};
  const int t0 = a.cta_start[blockIdx.x], t1 = a.cta_start[blockIdx.x + 1];
  const int n = t1 - t0;
  if (producer) {
    int prev_inst = -1, prev_end = -1, par = 0;
    for (int k = 0; k < n; ++k) {
      const TileTask tk = a.tiles[t0 + k];
      if (k >= 2) named_sync(kBarEmpty + (k & 1), NT);  // consumers are done with tile k-2
      if (tk.inst != acc.inst) {
        eacc_flush<ENERGY, TRACE>(a, acc);
        acc.inst = tk.inst;
      }
      if (k == 0) {  // the block's first tile with the consumer warps, which have nothing to solve yet
        produce(tk, 0, false, par, whole_block(), acc);
        __syncthreads();
      } else {
        produce(tk, k & 1, tk.inst == prev_inst && tk.j0 == prev_end, par, grp, acc);
        named_arrive(kBarFull + (k & 1), NT);
      }
      prev_inst = tk.inst;
      prev_end = tk.j0 + tk.nl;
      par ^= 1;
    }
    if (n >= 2) named_sync(kBarEmpty + (n & 1), NT);  // consumers are done with tile n-2
    if (n >= 1) {  // the last tile's stores with the consumer warps, once they have solved it
      __syncthreads();
      finish(a.tiles[t1 - 1], (n - 1) & 1, whole_block(), acc);
    }
  } else {
    for (int k = 0; k < n; ++k) {
      const TileTask tk = a.tiles[t0 + k];
      if (tk.inst != acc.inst) {
        eacc_flush<ENERGY, TRACE>(a, acc);
        acc.inst = tk.inst;
      }
      if (k == 0) {
        produce(tk, 0, false, 0, whole_block(), acc);
        __syncthreads();
      } else {
        named_sync(kBarFull + (k & 1), NT);
      }
      solve(tk, k & 1, grp);
      if (k == n - 1) {  // the last tile's stores with the producer warps, which are done
        __syncthreads();
        finish(tk, k & 1, whole_block(), acc);
      } else {
        grp.sync();  // the stores read every consumer warp's solutions
        finish(tk, k & 1, grp, acc);
        named_arrive(kBarEmpty + (k & 1), NT);
      }
    }
  }
}

// The same pipeline with the stores moved to the producers: consumers only
// solve (tile t after "full" t, then "solved" t), producers finish tile t
// (stores, trace, energy) before assembling tile t+2 into the same buffer.
// For the mixed step, whose FP32 rows and pair update are cheap next to its
// FP64 solves, this keeps the solving warps on the FP64 work alone.
template <bool ENERGY, bool TRACE, class Produce, class Solve, class Finish>
__device__ __forceinline__ void pipe_tiles_finish_by_producers(const StepArgs& a, EAcc& acc,
                                                                Produce produce, Solve solve,
                                                                Finish finish) {
  const int nw = blockDim.x >> 5, P = a.pipe_producers, C = nw - P, NT = blockDim.x;
  const bool producer = (int)(threadIdx.x >> 5) < P;
  const WarpGroup grp = producer ? WarpGroup{0, P, kBarProd} : WarpGroup{P, C, kBarCons};
  const int t0 = a.cta_start[blockIdx.x], t1 = a.cta_start[blockIdx.x + 1];
  const int n = t1 - t0;
  if (n == 0) return;
  auto use_inst = [&](int inst) {  // the energy and trace sums belong to one instance
    if (inst != acc.inst) {
      eacc_flush<ENERGY, TRACE>(a, acc);
      acc.inst = inst;
    }
  };
  // tile 0 with all warps (the consumers have nothing to solve yet)
  {
    const TileTask tk = a.tiles[t0];
    use_inst(tk.inst);
    produce(tk, 0, false, 0, whole_block(), acc);
    __syncthreads();
  }
  if (producer) {
    int prev_inst = a.tiles[t0].inst, prev_end = a.tiles[t0].j0 + a.tiles[t0].nl, par = 1;
    auto next = [&](int k) {  // assemble tile k into buffer k & 1, hand it to the consumers
      const TileTask tk = a.tiles[t0 + k];
      use_inst(tk.inst);
      produce(tk, k & 1, tk.inst == prev_inst && tk.j0 == prev_end, par, grp, acc);
      named_arrive(kBarFull + (k & 1), NT);
      prev_inst = tk.inst;
      prev_end = tk.j0 + tk.nl;
      par ^= 1;
    };
    if (n >= 2) next(1);
    for (int t = 0; t < n - 1; ++t) {
      named_sync(kBarSolved + (t & 1), NT);  // the consumers have solved tile t
      const TileTask tk = a.tiles[t0 + t];
      use_inst(tk.inst);
      finish(tk, t & 1, grp, acc);
      if (t + 2 < n) {
        grp.sync();  // every producer is done reading buffer t & 1
        next(t + 2);
      }
    }
  } else {
    for (int t = 0; t < n; ++t) {
      if (t >= 1) named_sync(kBarFull + (t & 1), NT);
      solve(a.tiles[t0 + t], t & 1, grp);
      if (t < n - 1) named_arrive(kBarSolved + (t & 1), NT);
    }
  }
  // the last tile's stores with all warps, once it is solved
  __syncthreads();
  const TileTask tk = a.tiles[t1 - 1];
  use_inst(tk.inst);
  finish(tk, (n - 1) & 1, whole_block(), acc);
}

template <bool ENERGY, bool TRACE>
__global__ void __launch_bounds__(384, 1) step_fp64_pipe_kernel(const StepArgs a) {
  extern __shared__ double sm[];
  double* buf0 = sm + 2 * kCarryStride;
  EAcc acc;
  eacc_init(acc);
  auto tile = [&](const TileTask& tk, int b) {
    const int nrp = smem_row_stride(a.insts[tk.inst].nr);
    return fp64_tile_at(buf0 + (size_t)b * a.pipe_buf, tk.nl, nrp);
  };
  pipe_tiles<ENERGY, TRACE>(
      a, acc,
      [&](const TileTask& tk, int b, bool carry, int par, const WarpGroup& grp, EAcc& ac) {
        const DevInst& I = a.insts[tk.inst];
        const int nrp = smem_row_stride(I.nr);
        const GlobalField<true> fld(a, I);
        if (tk.j0 + tk.nl >= I.j_narrow)
          fp64_produce<ENERGY, true>(a, tk, tile(tk, b), sm + (size_t)(par ^ 1) * nrp,
                                     sm + (size_t)par * nrp, carry, grp, ac, fld);
        else
          fp64_produce<ENERGY, false>(a, tk, tile(tk, b), sm + (size_t)(par ^ 1) * nrp,
                                      sm + (size_t)par * nrp, carry, grp, ac, fld);
      },
      [&](const TileTask& tk, int b, const WarpGroup& grp) {
        const DevInst& I = a.insts[tk.inst];
        const Fp64Tile B = tile(tk, b);
        solve_tile_lines<true>(B.SA, B.SB, B.SC, B.SD, tk.nl, I.nr, I.G, grp.warp());
      },
      [&](const TileTask& tk, int b, const WarpGroup& grp, EAcc& ac) {
        const DevInst& I = a.insts[tk.inst];
        const Fp64Tile B = tile(tk, b);
        const GlobalField<true> fld(a, I);
        if (tk.j0 + tk.nl >= I.j_narrow)
          fp64_finish<ENERGY, TRACE, true>(a, tk, B, grp, ac, fld);
        else
          fp64_finish<ENERGY, TRACE, false>(a, tk, B, grp, ac, fld);
      });
  eacc_flush<ENERGY, TRACE>(a, acc);
}

// MAXT: the largest block the variant is compiled for (its register budget:
// 384 threads leave about 170 registers a thread, 512 threads 128).  STORES:
// the producers store every tile (launch mode 5) instead of the consumers
// (launch mode 4).
template <bool ENERGY, bool TRACE, int MAXT, bool STORES>
__global__ void __launch_bounds__(MAXT, 1) step_mixed_pipe_kernel(const StepArgs a) {
  extern __shared__ float4 smq[];
  float* smf = reinterpret_cast<float*>(smq);
  float* buf0 = smf + kCarryFloats;
  EAcc acc;
  eacc_init(acc);
  auto tile = [&](const TileTask& tk, int b) {  // packed rows
    const int nrp = smem_row_stride(a.insts[tk.inst].nr);
    return mix_tile_packed_at(buf0 + (size_t)b * a.pipe_buf, tk.nl, nrp);
  };
  auto produce = [&](const TileTask& tk, int b, bool carry, int par, const WarpGroup& grp,
                     EAcc& ac) {
        const DevInst& I = a.insts[tk.inst];
        const int nrp = smem_row_stride(I.nr);
        if (tk.j0 + tk.nl >= I.j_narrow)
          mixed_produce<ENERGY, true, true, true>(a, tk, tile(tk, b), smf + (size_t)(par ^ 1) * nrp,
                                                  smf + (size_t)par * nrp, carry, grp, ac);
        else
          mixed_produce<ENERGY, true, false, true>(a, tk, tile(tk, b), smf + (size_t)(par ^ 1) * nrp,
                                                   smf + (size_t)par * nrp, carry, grp, ac);
      };
  auto solve = [&](const TileTask& tk, int b, const WarpGroup& grp) {
        const DevInst& I = a.insts[tk.inst];
        solve_mixed_packed(tile(tk, b).Q, tk.nl, I.nr, I.G, grp.warp());
      };
  auto finish = [&](const TileTask& tk, int b, const WarpGroup& grp, EAcc& ac) {
        const DevInst& I = a.insts[tk.inst];
        const MixTile B = tile(tk, b);
        if (tk.j0 + tk.nl >= I.j_narrow)
          mixed_finish<ENERGY, TRACE, true, true, true>(a, tk, B, grp, ac);
        else
          mixed_finish<ENERGY, TRACE, true, false, true>(a, tk, B, grp, ac);
      };
  if constexpr (STORES)
    pipe_tiles_finish_by_producers<ENERGY, TRACE>(a, acc, produce, solve, finish);
  else
    pipe_tiles<ENERGY, TRACE>(a, acc, produce, solve, finish);
  eacc_flush<ENERGY, TRACE>(a, acc);
}

template <bool ENERGY, bool TRACE>
static KernelCache& fp64_pipe_cache() {
  static KernelCache c;
  return c;
}
template <bool ENERGY, bool TRACE, int MAXT, bool STORES>
static KernelCache& mixed_pipe_cache() {
  static KernelCache c;
  return c;
}

template <bool ENERGY, bool TRACE, bool STORES>
static int mixed_variant_resident(int threads, int smem) {
  if (threads > 384)
    return cached_resident(mixed_pipe_cache<ENERGY, TRACE, 512, STORES>(),
                           step_mixed_pipe_kernel<ENERGY, TRACE, 512, STORES>, threads, smem,
                           kMaxTileSmem);
  return cached_resident(mixed_pipe_cache<ENERGY, TRACE, 384, STORES>(),
                         step_mixed_pipe_kernel<ENERGY, TRACE, 384, STORES>, threads, smem,
                         kMaxTileSmem);
}

template <bool MIXED, bool ENERGY, bool TRACE>
static int pipe_variant_resident(int threads, int smem) {
  if constexpr (MIXED) {
    return min(mixed_variant_resident<ENERGY, TRACE, false>(threads, smem),
               mixed_variant_resident<ENERGY, TRACE, true>(threads, smem));
  } else {
    return cached_resident(fp64_pipe_cache<ENERGY, TRACE>(), step_fp64_pipe_kernel<ENERGY, TRACE>,
                           threads, smem, kMaxTileSmem);
  }
}

template <bool MIXED>
static int pipe_resident(int threads, int smem) {
  int r = pipe_variant_resident<MIXED, true, true>(threads, smem);
  r = min(r, pipe_variant_resident<MIXED, true, false>(threads, smem));
  r = min(r, pipe_variant_resident<MIXED, false, true>(threads, smem));
  return min(r, pipe_variant_resident<MIXED, false, false>(threads, smem));
}
int fp64_pipe_resident_blocks(int threads, int smem) { return pipe_resident<false>(threads, smem); }
int mixed_pipe_resident_blocks(int threads, int smem) { return pipe_resident<true>(threads, smem); }

template <bool MIXED, bool ENERGY, bool TRACE>
static int launch_pipe_variant(const StepArgs& a, cudaStream_t st) {
  if (pipe_variant_resident<MIXED, ENERGY, TRACE>(a.threads, a.smem_bytes) < 0) return -1;
  if constexpr (MIXED) {
    if (a.threads > 384) {
      if (a.pipe_stores)
        step_mixed_pipe_kernel<ENERGY, TRACE, 512, true><<<a.n_cta, a.threads, a.smem_bytes, st>>>(a);
      else
        step_mixed_pipe_kernel<ENERGY, TRACE, 512, false><<<a.n_cta, a.threads, a.smem_bytes, st>>>(a);
    } else {
      if (a.pipe_stores)
        step_mixed_pipe_kernel<ENERGY, TRACE, 384, true><<<a.n_cta, a.threads, a.smem_bytes, st>>>(a);
      else
        step_mixed_pipe_kernel<ENERGY, TRACE, 384, false><<<a.n_cta, a.threads, a.smem_bytes, st>>>(a);
    }
  } else
    step_fp64_pipe_kernel<ENERGY, TRACE><<<a.n_cta, a.threads, a.smem_bytes, st>>>(a);
  return 0;
}

template <bool MIXED>
static int launch_pipe(const StepArgs& a, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const bool E = a.energy != nullptr, T = a.trace != nullptr;
  int r;
  if (E && T) r = launch_pipe_variant<MIXED, true, true>(a, st);
  else if (E) r = launch_pipe_variant<MIXED, true, false>(a, st);
  else if (T) r = launch_pipe_variant<MIXED, false, true>(a, st);
  else r = launch_pipe_variant<MIXED, false, false>(a, st);
  count_launch();
  if (r) return r;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_step_fp64_pipe(const StepArgs& a, void* stream) { return launch_pipe<false>(a, stream); }
int launch_step_mixed_pipe(const StepArgs& a, void* stream) { return launch_pipe<true>(a, stream); }

}  // namespace ccell
