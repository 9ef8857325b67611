// DEG and FAN of every edge, one window and direction (Sec. 5: DEG and FAN
// stages over a trailing window of the edge's own account).
//
// DEG(p) = p - lb(p) + 1 for slot p of a row sorted by (t, id), lb(p) the
// first slot of the row inside [t_p - delta, t_p].  FAN(p) = DEG(p) - R(p),
// R(p) the repeats in the window (slots whose previous same-counterparty
// slot is also inside).  R is a per-row prefix sum of the deltas
//   R(p) - R(p-1) = [prev(p) >= lb(p)] - #{r in [lb(p-1), lb(p)) : next(r) <= p-1}
// (the window gains p and drops [lb(p-1), lb(p))), with R(row start) = 0.
//
// Two launches over contiguous chunks of slots:
//   k_fan_reduce (a thread per slot, a block per chunk of FAN_RBLOCK): lb,
//     DEG and the delta of every slot, and per chunk the sum of the deltas
//     after its last row start (all of them when no row starts inside) with
//     a flag telling whether a row starts inside;
//   k_fan_scan (a block per tile of FAN_TILE slots): the carry into its tile
//     from those chunk sums (back to the nearest chunk where a row starts),
//     then a segmented scan of the deltas (restarting at row starts), and
//     (DEG, FAN) stored at the edge id of every slot.
#include <algorithm>

#include "aml_internal.cuh"
#include "mine.cuh"
#include "profile.cuh"

namespace aml {

namespace {

constexpr int FAN_RBLOCK = 512;  // slots per k_fan_reduce block (one each)
constexpr int FAN_BLOCK = 256;
constexpr int FAN_ITEMS = 8;
constexpr int FAN_TILE = FAN_BLOCK * FAN_ITEMS;
constexpr int FAN_SMEM = FAN_TILE + FAN_TILE / 32;  // one pad word per 32

__device__ __forceinline__ int fpad(int i) { return i + (i >> 5); }

// segmented-sum pair: h = a row starts in the range, v = sum of the values
// after (and at) its last row start, or of all of them when h = 0
struct Seg {
  int32_t h, v;
};
__device__ __forceinline__ Seg seg_combine(Seg a, Seg b) {  // a, then b
  return Seg{a.h | b.h, b.h ? b.v : a.v + b.v};
}

// exclusive segmented scan of one pair per thread over the block, in thread
// order; *total = the block's combined pair
__device__ Seg seg_scan_block(Seg x, Seg* total) {
  __shared__ Seg s_w[FAN_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Seg inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Seg y;
    y.h = __shfl_up_sync(0xffffffffu, inc.h, o);
    y.v = __shfl_up_sync(0xffffffffu, inc.v, o);
    if (lane >= o) inc = seg_combine(y, inc);
  }
  Seg ex;
  ex.h = __shfl_up_sync(0xffffffffu, inc.h, 1);
  ex.v = __shfl_up_sync(0xffffffffu, inc.v, 1);
  if (lane == 0) ex = Seg{0, 0};
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    Seg w = lane < FAN_BLOCK / 32 ? s_w[lane] : Seg{0, 0};
#pragma unroll
    for (int o = 1; o < FAN_BLOCK / 32; o <<= 1) {
      Seg y;
      y.h = __shfl_up_sync(0xffffffffu, w.h, o);
      y.v = __shfl_up_sync(0xffffffffu, w.v, o);
      if (lane >= o) w = seg_combine(y, w);
    }
    if (lane < FAN_BLOCK / 32) s_w[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const Seg before = warp ? s_w[warp - 1] : Seg{0, 0};
  *total = s_w[FAN_BLOCK / 32 - 1];
  const Seg r = seg_combine(before, ex);
  __syncthreads();  // s_w is reused by the next call
  return r;
}

// one slot per thread; chunks of FAN_RBLOCK slots
__global__ void __launch_bounds__(FAN_RBLOCK) k_fan_reduce(const int32_t* __restrict__ rstart,
                                                           const int32_t* __restrict__ t,
                                                           const int32_t* __restrict__ prev,
                                                           const int32_t* __restrict__ next,
                                                           int64_t Ev, int32_t delta,
                                                           int32_t* __restrict__ deg_s,
                                                           int32_t* __restrict__ D,
                                                           int2* __restrict__ chunk_sum) {
  __shared__ int32_t s_sum[FAN_RBLOCK / 32];
  const int lane = threadIdx.x & 31;
  const int64_t c0 = (int64_t)blockIdx.x * FAN_RBLOCK;
  const int64_t c1 = c0 + FAN_RBLOCK < Ev ? c0 + FAN_RBLOCK : Ev;
  const int32_t last_rs = rstart[c1 - 1];  // the last row start at or before the chunk's end
  const int64_t from = last_rs > c0 ? last_rs : c0;
  const int64_t p64 = c0 + threadIdx.x;
  const bool in = p64 < c1;
  const int32_t p = (int32_t)p64;
  int32_t rs = 0, lbp = 0, u = 0;
  if (in) {
    rs = __ldg(rstart + p);
    lbp = lower_t(t, rs, p + 1, (int64_t)__ldg(t + p) - delta);
    deg_s[p] = p - lbp + 1;
  }
  // lb(p-1) is the lower lane's lb when that lane holds slot p-1 of the row
  const int32_t lb_lower = __shfl_up_sync(0xffffffffu, lbp, 1);
  if (in) {
    int32_t d = 0;
    if (p > rs) {
      const int32_t lbq =
          lane > 0 ? lb_lower
                   : lower_t(t, rs, min(lbp + 1, p), (int64_t)__ldg(t + p - 1) - delta);
      d = (__ldg(prev + p) >= lbp) ? 1 : 0;
      for (int32_t r = lbq; r < lbp; ++r) d -= (__ldg(next + r) <= p - 1) ? 1 : 0;
    }
    D[p] = d;
    if (p64 >= from) u = d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
  if (lane == 0) s_sum[threadIdx.x >> 5] = u;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t tot = 0;
    for (int w = 0; w < FAN_RBLOCK / 32; ++w) tot += s_sum[w];
    chunk_sum[blockIdx.x] = make_int2(tot, last_rs >= c0 ? 1 : 0);
  }
}

__global__ void __launch_bounds__(FAN_BLOCK) k_fan_scan(const int32_t* __restrict__ rstart,
                                                        const int32_t* __restrict__ eid,
                                                        const int32_t* __restrict__ deg_s,
                                                        const int32_t* __restrict__ D,
                                                        int64_t Ev,
                                                        const int2* __restrict__ chunk_sum,
                                                        int2* __restrict__ df) {
  __shared__ int32_t s_v[FAN_SMEM];
  __shared__ uint8_t s_h[FAN_SMEM];
  __shared__ int32_t s_carry;
  const int64_t c0 = (int64_t)blockIdx.x * FAN_TILE;
  const int64_t c1 = c0 + FAN_TILE < Ev ? c0 + FAN_TILE : Ev;
  if (threadIdx.x < 32) {
    // deltas of the row running into the tile: the sums of the reduce
    // chunks before it back to the nearest one where a row starts (chunk 0
    // always has one: slot 0), 32 chunks per step
    const int lane = threadIdx.x;
    int32_t v = 0;
    for (int64_t top = c0 / FAN_RBLOCK - 1; top >= 0; top -= 32) {
      const int64_t c = top - lane;
      const int2 cs = c >= 0 ? chunk_sum[c] : make_int2(0, 1);
      const unsigned starts = __ballot_sync(0xffffffffu, cs.y != 0);
      const int first = starts ? __ffs(starts) - 1 : 31;  // lanes [0, first] count
      int32_t x = lane <= first ? cs.x : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v += x;
      if (starts) break;
    }
    if (lane == 0) s_carry = v;
  }
  __syncthreads();
  Seg run{0, s_carry};
  for (int64_t base = c0; base < c1; base += FAN_TILE) {
    for (int i = threadIdx.x; i < FAN_TILE; i += FAN_BLOCK) {
      const int64_t p = base + i;
      const bool in = p < c1;
      s_v[fpad(i)] = in ? D[p] : 0;
      s_h[fpad(i)] = in && rstart[p] == (int32_t)p ? 1 : 0;
    }
    __syncthreads();
    int32_t v[FAN_ITEMS];
    uint8_t h[FAN_ITEMS];
    Seg mine{0, 0};
#pragma unroll
    for (int k = 0; k < FAN_ITEMS; ++k) {
      const int j = fpad(threadIdx.x * FAN_ITEMS + k);
      v[k] = s_v[j];
      h[k] = s_h[j];
      mine = seg_combine(mine, Seg{h[k], v[k]});
    }
    Seg tile_total;
    const Seg ex = seg_scan_block(mine, &tile_total);
    int32_t r = seg_combine(run, ex).v;
#pragma unroll
    for (int k = 0; k < FAN_ITEMS; ++k) {
      r = h[k] ? v[k] : r + v[k];
      s_v[fpad(threadIdx.x * FAN_ITEMS + k)] = r;  // R of the slot
    }
    __syncthreads();
    for (int i = threadIdx.x; i < FAN_TILE; i += FAN_BLOCK) {
      const int64_t p = base + i;
      if (p < c1) {
        const int32_t deg = deg_s[p];
        df[eid[p]] = make_int2(deg, deg - s_v[fpad(i)]);
      }
    }
    run = seg_combine(run, tile_total);
    __syncthreads();  // s_v / s_h are refilled by the next tile
  }
}

}  // namespace

void fan_per_edge(const Adj& a, int64_t Ev, int32_t delta, int2* df, cudaStream_t s) {
  if (Ev <= 0) return;
  const int64_t n_red = (Ev + FAN_RBLOCK - 1) / FAN_RBLOCK;
  const int64_t n_tiles = (Ev + FAN_TILE - 1) / FAN_TILE;
  DBuf<int32_t> deg_s((size_t)Ev, s), D((size_t)Ev, s);
  DBuf<int2> sums((size_t)n_red, s);
  AML_LAUNCH("k_fan_reduce", s,
             k_fan_reduce<<<(unsigned)n_red, FAN_RBLOCK, 0, s>>>(a.rstart, a.t, a.prev, a.next,
                                                                 Ev, delta, deg_s.p, D.p,
                                                                 sums.p));
  AML_LAUNCH("k_fan_scan", s,
             k_fan_scan<<<(unsigned)n_tiles, FAN_BLOCK, 0, s>>>(a.rstart, a.eid, deg_s.p, D.p,
                                                                Ev, sums.p, df));
}

}  // namespace aml
