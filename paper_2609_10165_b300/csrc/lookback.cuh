// Block-level and single-pass device-wide exclusive scans of int32 counts
// (stream compaction offsets).
//
// Single pass: every block takes its tile index from a ticket counter, so a
// tile only ever waits on tiles whose blocks are already running.  It
// publishes its aggregate, then its threads read the published aggregates of
// all tiles before it in parallel (a strided share each) and the block adds
// them up.  No tile waits on another tile's prefix, so there is no chain of
// waits: the usual decoupled look-back, which walks back one predecessor at a
// time, degenerates into such a chain when all tiles of a one-wave grid start
// together.  A few thousand tiles at most here, so the reads (tiles^2 / 2
// words from L2) are cheap.  Integer sums: the offsets are those of a
// sequential scan in tile order.
//
// State (device memory, zeroed once when allocated):
//   ctr[0] ticket, ctr[1] epoch, ctr[2] blocks finished;
//   tiles[t] = epoch (30 bits) << 34 | published (2 bits) << 32 | aggregate.
// The last block of a launch to finish resets the ticket and the finished
// count and advances the epoch, so that the next launch reads every word of
// this one as not yet published.  Two launches must not use one state at the
// same time (each user has its own, on one stream).
//
// Every wait is bounded: after `spin_limit` polls of one word the block
// records EBR_ETIMEOUT and writes nothing.  In a correct run every
// predecessor publishes, since it holds a smaller ticket, is running, and
// publishes before it reads anything.
#pragma once

#include "ebr_device.cuh"

namespace ebr {

constexpr int LB_T = 256;   // threads (items) per tile of the single-pass kernels

// exclusive scan of one int per thread over the block; total = block sum.
// Every thread of the block must call it.
__device__ inline int block_excl_scan(int v, int* sh_warp, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    int s = lane < nw ? sh_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sh_warp[lane] = s;
  }
  __syncthreads();
  int before = w > 0 ? sh_warp[w - 1] : 0;
  total = sh_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

struct Lookback {
  unsigned* ctr;                 // [3]
  unsigned long long* tiles;     // [n_tiles]
  int spin_limit;
};

constexpr unsigned LB_AGG = 1u;   // a published aggregate

__device__ __forceinline__ unsigned long long lb_pack(unsigned epoch, unsigned state, unsigned value) {
  return ((unsigned long long)(epoch & 0x3FFFFFFFu) << 34) | ((unsigned long long)state << 32) | value;
}

// A tile word carries its own data (epoch, state and value in one 64-bit
// access), so the polls need no ordering with other memory: relaxed
// device-scope accesses (acquire loads would order, and cost, every poll)
__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Per-block state of one single-pass scan.
struct LbBlock {
  int tile;
  unsigned epoch;
};

// Tile index of this block (ticket order) and the launch's epoch.  Every
// thread of the block must call it; it synchronises the block.
__device__ inline LbBlock lb_begin(const Lookback& L) {
  __shared__ int s_tile;
  __shared__ unsigned s_epoch;
  if (threadIdx.x == 0) {
    s_tile = (int)atomicAdd(&L.ctr[0], 1u);
    s_epoch = atomicAdd(&L.ctr[1], 0u);
  }
  __syncthreads();
  LbBlock b;
  b.tile = s_tile;
  b.epoch = s_epoch;
  return b;
}

// Exclusive prefix of this tile: the sum of the aggregates of all tiles
// before it.  agg = the block's total.  Returns -1 when a wait gave up (the
// caller then writes nothing).  Every thread of the block must call it.
__device__ inline long long lb_prefix(const Lookback& L, const LbBlock& b, unsigned agg, int* status) {
  __shared__ long long s_part[32];
  if (threadIdx.x == 0) lb_store(&L.tiles[b.tile], lb_pack(b.epoch, LB_AGG, agg));
  const unsigned e = b.epoch & 0x3FFFFFFFu;
  long long part = 0;
  int bad = 0;
  for (int p = threadIdx.x; p < b.tile && !bad; p += blockDim.x) {
    for (int spins = 0;; ++spins) {
      const unsigned long long w = lb_load(&L.tiles[p]);
      if ((unsigned)(w >> 34) == e && ((unsigned)(w >> 32) & 3u) != 0u) {
        part += (long long)(unsigned)w;
        break;
      }
      if (spins >= L.spin_limit) { bad = 1; break; }
      __nanosleep(64);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) s_part[warp] = part;
  bad = __syncthreads_or(bad);
  if (bad) {
    if (threadIdx.x == 0) set_status(status, S_ETIMEOUT);
    return -1;
  }
  long long sum = 0;
  for (int w = 0; w < nw; ++w) sum += s_part[w];
  if (sum + agg > 0xFFFFFFFFll) {
    if (threadIdx.x == 0) set_status(status, S_ESHAPE);
    return -1;
  }
  return sum;
}

// End of the block's part: the last block of the launch resets the state for
// the next launch.  Every thread of the block must call it, after its writes.
__device__ inline void lb_end(const Lookback& L) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&L.ctr[2], 1u);
    if (done == gridDim.x - 1) {
      atomicExch(&L.ctr[0], 0u);
      atomicExch(&L.ctr[2], 0u);
      atomicAdd(&L.ctr[1], 1u);
    }
  }
}

}  // namespace ebr
