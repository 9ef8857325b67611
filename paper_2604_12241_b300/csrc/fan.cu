// DEG and FAN of every edge for up to FAN_MAX_W windows of one direction
// (Sec. 5: DEG and FAN stages over a trailing window of the edge's own
// account).
//
// DEG(p) = p - lb(p) + 1 for slot p of a row sorted by (t, id), lb(p) the
// first slot of the row inside [t_p - delta, t_p].  FAN(p) = DEG(p) - R(p),
// R(p) the repeats in the window (slots whose previous same-counterparty
// slot is also inside).  R is a per-row prefix sum of the deltas
//   R(p) - R(p-1) = [prev(p) >= lb(p)] - #{r in [lb(p-1), lb(p)) : next(r) <= p-1}
// (the window gains p and drops [lb(p-1), lb(p))), with R(row start) = 0.
//
// Two launches over tiles of FAN_TILE consecutive slots (a block each), all
// W windows at once (the windows are nested, so each window start is
// searched above the previous one, and the W results of an edge leave in
// one store):
//   k_fan_reduce: lb, DEG and the delta of every slot (two pointers along
//     FAN_ITEMS consecutive slots per thread), and per tile the sum of the
//     deltas after its last row start (all of them when no row starts
//     inside) with a flag telling whether a row starts inside;
//   k_fan_scan: the carry into its tile from those tile sums (back to the
//     nearest tile where a row starts), then a segmented scan of the deltas
//     (restarting at row starts), and (DEG, FAN) of every window stored at
//     the edge id of every slot.
#include <algorithm>
#include <type_traits>

#include "aml_internal.cuh"
#include "mine.cuh"
#include "profile.cuh"

namespace aml {

namespace {

constexpr int FAN_BLOCK = 256;
constexpr int FAN_ITEMS = 4;                         // slots per thread of k_fan_reduce
constexpr int FAN_TILE = FAN_BLOCK * FAN_ITEMS;      // slots per block (chunk sums)
constexpr int SCAN_ITEMS = 4;                        // slots per thread of a scan pass
constexpr int SCAN_TILE = FAN_BLOCK * SCAN_ITEMS;    // a chunk is scanned in passes of this
constexpr int FAN_SMEM = SCAN_TILE + SCAN_TILE / 32;  // one pad word per 32

__device__ __forceinline__ int fpad(int i) { return i + (i >> 5); }

struct FanDeltas {
  int32_t d[FAN_MAX_W];  // descending
};

// segmented sums: h = a row starts in the range, v[k] = sum of the values
// after (and at) its last row start, or of all of them when h = 0
template <int W>
struct Seg {
  int32_t h;
  int32_t v[W];
};
template <int W>
__device__ __forceinline__ Seg<W> seg_combine(const Seg<W>& a, const Seg<W>& b) {  // a, then b
  Seg<W> r;
  r.h = a.h | b.h;
#pragma unroll
  for (int k = 0; k < W; ++k) r.v[k] = b.h ? b.v[k] : a.v[k] + b.v[k];
  return r;
}
template <int W>
__device__ __forceinline__ Seg<W> seg_shfl_up(const Seg<W>& x, int o) {
  Seg<W> y;
  y.h = __shfl_up_sync(0xffffffffu, x.h, o);
#pragma unroll
  for (int k = 0; k < W; ++k) y.v[k] = __shfl_up_sync(0xffffffffu, x.v[k], o);
  return y;
}
template <int W>
__device__ __forceinline__ Seg<W> seg_zero() {
  Seg<W> z;
  z.h = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) z.v[k] = 0;
  return z;
}

// exclusive segmented scan of one value set per thread over the block, in
// thread order; *total = the block's combined set
template <int W>
__device__ Seg<W> seg_scan_block(const Seg<W>& x, Seg<W>* total) {
  __shared__ Seg<W> s_w[FAN_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Seg<W> inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Seg<W> y = seg_shfl_up(inc, o);
    if (lane >= o) inc = seg_combine(y, inc);
  }
  Seg<W> ex = seg_shfl_up(inc, 1);
  if (lane == 0) ex = seg_zero<W>();
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    Seg<W> w = lane < FAN_BLOCK / 32 ? s_w[lane] : seg_zero<W>();
#pragma unroll
    for (int o = 1; o < FAN_BLOCK / 32; o <<= 1) {
      const Seg<W> y = seg_shfl_up(w, o);
      if (lane >= o) w = seg_combine(y, w);
    }
    if (lane < FAN_BLOCK / 32) s_w[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const Seg<W> before = warp ? s_w[warp - 1] : seg_zero<W>();
  *total = s_w[FAN_BLOCK / 32 - 1];
  const Seg<W> r = seg_combine(before, ex);
  __syncthreads();  // s_w is reused by the next call
  return r;
}

// deg_s, D: [W][Ev]; chunk_sum: [W][n_tiles].  Thread t of block b walks
// the FAN_ITEMS consecutive slots from b * FAN_TILE + t * FAN_ITEMS: one
// binary search per window for the slot before its first slot, then every
// window start only moves forward (two pointers), and the slots it passes
// are exactly the dropped range of the repeat delta.
template <int W>
__global__ void __launch_bounds__(FAN_BLOCK) k_fan_reduce(const int32_t* __restrict__ rstart,
                                                          const int32_t* __restrict__ t,
                                                          const int32_t* __restrict__ prev,
                                                          const int32_t* __restrict__ next,
                                                          int64_t Ev, FanDeltas fd,
                                                          int32_t* __restrict__ deg_s,
                                                          int32_t* __restrict__ D,
                                                          int2* __restrict__ chunk_sum) {
  __shared__ int32_t s_sum[W][FAN_BLOCK / 32];
  const int lane = threadIdx.x & 31;
  const int64_t c0 = (int64_t)blockIdx.x * FAN_TILE;
  const int64_t c1 = c0 + FAN_TILE < Ev ? c0 + FAN_TILE : Ev;
  const int32_t last_rs = rstart[c1 - 1];  // the last row start at or before the chunk's end
  const int64_t from = last_rs > c0 ? last_rs : c0;
  const int64_t p0 = c0 + (int64_t)threadIdx.x * FAN_ITEMS;
  const int64_t p1 = p0 + FAN_ITEMS < c1 ? p0 + FAN_ITEMS : c1;
  int32_t u[W];
#pragma unroll
  for (int k = 0; k < W; ++k) u[k] = 0;
  if (p0 < p1) {
    // window starts of slot p0 - 1 when it lies in p0's row
    int32_t lb[W];
    const int32_t rs0 = __ldg(rstart + p0);
    if (p0 > rs0) {
      const int64_t tq = __ldg(t + p0 - 1);
      int32_t lo = rs0;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        lb[k] = lower_t(t, lo, (int32_t)p0, tq - fd.d[k]);  // nested: lb grows
        lo = lb[k];
      }
    }
    for (int64_t p64 = p0; p64 < p1; ++p64) {
      const int32_t p = (int32_t)p64;
      const bool head = __ldg(rstart + p) == p;
      const int64_t tp = __ldg(t + p);
      const int32_t pv = head ? -1 : __ldg(prev + p);
#pragma unroll
      for (int k = 0; k < W; ++k) {
        int32_t d = 0;
        if (head) {
          lb[k] = p;
        } else {
          int32_t l = lb[k], gone = 0;
          const int64_t tmin = tp - fd.d[k];
          while (__ldg(t + l) < tmin) {  // stops at p at the latest: t[p] >= tmin
            gone += __ldg(next + l) <= p - 1 ? 1 : 0;
            ++l;
          }
          lb[k] = l;
          d = (pv >= l ? 1 : 0) - gone;
        }
        deg_s[k * Ev + p] = p - lb[k] + 1;
        D[k * Ev + p] = d;
        if (p64 >= from) u[k] += d;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < W; ++k) {
    int32_t x = u[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_sum[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < W) {
    const int k = threadIdx.x;
    int32_t tot = 0;
    for (int w = 0; w < FAN_BLOCK / 32; ++w) tot += s_sum[k][w];
    chunk_sum[(int64_t)k * gridDim.x + blockIdx.x] = make_int2(tot, last_rs >= c0 ? 1 : 0);
  }
}

// edge e's row of df: the W (DEG, FAN) pairs and zero padding, 32 bytes in
// two 16-byte stores (a whole sector, so no read-modify-write)
template <int W>
__device__ __forceinline__ void store_df(int2* __restrict__ df, int32_t e, const int2 (&v)[W]) {
  static_assert(W <= DF_STRIDE, "window count");
  int2 r[DF_STRIDE];
#pragma unroll
  for (int k = 0; k < DF_STRIDE; ++k) r[k] = k < W ? v[k] : make_int2(0, 0);
  int4* dst = reinterpret_cast<int4*>(df + (int64_t)e * DF_STRIDE);
  dst[0] = make_int4(r[0].x, r[0].y, r[1].x, r[1].y);
  dst[1] = make_int4(r[2].x, r[2].y, r[3].x, r[3].y);
}

// df: [E][DF_STRIDE] (DEG, FAN) pairs in edge order, one whole 32-byte row
// per edge
template <int W>
__global__ void __launch_bounds__(FAN_BLOCK) k_fan_scan(const int32_t* __restrict__ rstart,
                                                        const int32_t* __restrict__ eid,
                                                        const int32_t* __restrict__ deg_s,
                                                        const int32_t* __restrict__ D,
                                                        int64_t Ev, int64_t n_tiles,
                                                        const int2* __restrict__ chunk_sum,
                                                        int2* __restrict__ df) {
  __shared__ int32_t s_v[W][FAN_SMEM];
  __shared__ uint8_t s_h[FAN_SMEM];
  __shared__ int32_t s_carry[W];
  const int64_t c0 = (int64_t)blockIdx.x * FAN_TILE;
  const int64_t c1 = c0 + FAN_TILE < Ev ? c0 + FAN_TILE : Ev;
  if (threadIdx.x < 32) {
    // deltas of the row running into the tile: the sums of the tiles before
    // it back to the nearest one where a row starts (tile 0 always has one:
    // slot 0), 32 tiles per step
    const int lane = threadIdx.x;
    int32_t v[W];
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = 0;
    for (int64_t top = (int64_t)blockIdx.x - 1; top >= 0; top -= 32) {
      const int64_t c = top - lane;
      const int32_t flag = c >= 0 ? chunk_sum[c].y : 1;
      const unsigned starts = __ballot_sync(0xffffffffu, flag != 0);
      const int first = starts ? __ffs(starts) - 1 : 31;  // lanes [0, first] count
#pragma unroll
      for (int k = 0; k < W; ++k) {
        int32_t x = (c >= 0 && lane <= first) ? chunk_sum[k * n_tiles + c].x : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        v[k] += x;
      }
      if (starts) break;
    }
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < W; ++k) s_carry[k] = v[k];
  }
  __syncthreads();
  Seg<W> run;
  run.h = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) run.v[k] = s_carry[k];
  for (int64_t base = c0; base < c1; base += SCAN_TILE) {
    for (int i = threadIdx.x; i < SCAN_TILE; i += FAN_BLOCK) {
      const int64_t p = base + i;
      const bool in = p < c1;
#pragma unroll
      for (int k = 0; k < W; ++k) s_v[k][fpad(i)] = in ? D[k * Ev + p] : 0;
      s_h[fpad(i)] = in && rstart[p] == (int32_t)p ? 1 : 0;
    }
    __syncthreads();
    Seg<W> mine = seg_zero<W>();
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; ++it) {
      const int j = fpad(threadIdx.x * SCAN_ITEMS + it);
      Seg<W> x;
      x.h = s_h[j];
#pragma unroll
      for (int k = 0; k < W; ++k) x.v[k] = s_v[k][j];
      mine = seg_combine(mine, x);
    }
    Seg<W> tile_total;
    const Seg<W> ex = seg_scan_block(mine, &tile_total);
    Seg<W> r = seg_combine(run, ex);
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; ++it) {
      const int j = fpad(threadIdx.x * SCAN_ITEMS + it);
      const bool h = s_h[j] != 0;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        r.v[k] = h ? s_v[k][j] : r.v[k] + s_v[k][j];
        s_v[k][j] = r.v[k];  // R of the slot
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += FAN_BLOCK) {
      const int64_t p = base + i;
      if (p < c1) {
        int2 v[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const int32_t deg = deg_s[k * Ev + p];
          v[k] = make_int2(deg, deg - s_v[k][fpad(i)]);
        }
        store_df<W>(df, __ldg(eid + p), v);
      }
    }
    run = seg_combine(run, tile_total);
    __syncthreads();  // s_v / s_h are refilled by the next tile
  }
}

template <int W>
void fan_launch(const Adj& a, int64_t Ev, const FanDeltas& fd, int2* df, cudaStream_t s) {
  const int64_t n_tiles = (Ev + FAN_TILE - 1) / FAN_TILE;
  DBuf<int32_t> deg_s((size_t)W * Ev, s), D((size_t)W * Ev, s);
  DBuf<int2> sums((size_t)W * n_tiles, s);
  AML_LAUNCH("k_fan_reduce", s,
             k_fan_reduce<W><<<(unsigned)n_tiles, FAN_BLOCK, 0, s>>>(
                 a.rstart, a.t, a.prev, a.next, Ev, fd, deg_s.p, D.p, sums.p));
  AML_LAUNCH("k_fan_scan", s,
             k_fan_scan<W><<<(unsigned)n_tiles, FAN_BLOCK, 0, s>>>(a.rstart, a.eid, deg_s.p, D.p,
                                                                   Ev, n_tiles, sums.p, df));
}

// ----------------------------------------------------------- batch rows
//
// Delta counting needs DEG/FAN only for the new edges (ids >= new_from),
// which are the last slots of their rows (they come after every older edge
// in the (t, id) order).  One block per row holding new slots: its threads
// count the distinct counterparties of the first new slot's windows
// directly (slots whose previous same-counterparty slot lies before the
// window start; a hub's window holds tens of thousands of slots), then one
// thread walks the row's remaining new slots with the repeat-delta
// recurrence (two pointers).

// first new slot of every row that has one: rows[*n_rows++]
__global__ void __launch_bounds__(256) k_batch_rows(const int32_t* __restrict__ pos,
                                                    const int32_t* __restrict__ rstart,
                                                    const int32_t* __restrict__ eid,
                                                    int64_t new_from, int64_t E,
                                                    int32_t* __restrict__ rows,
                                                    unsigned int* __restrict__ n_rows) {
  const int64_t e = new_from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t p = pos[e];
  if (p < 0) return;  // self-loop
  if (p == rstart[p] || eid[p - 1] < new_from) rows[atomicAdd(n_rows, 1u)] = p;
}

constexpr int FAN_BATCH_BLOCK = 128;

template <int W>
__global__ void __launch_bounds__(FAN_BATCH_BLOCK) k_fan_batch(const int32_t* __restrict__ rstart,
                                                   const int32_t* __restrict__ t,
                                                   const int32_t* __restrict__ eid,
                                                   const int32_t* __restrict__ prev,
                                                   const int32_t* __restrict__ next, int64_t Ev,
                                                   FanDeltas fd, const int32_t* __restrict__ rows,
                                                   const unsigned int* __restrict__ n_rows,
                                                   int2* __restrict__ df) {
  __shared__ int32_t s_c[FAN_BATCH_BLOCK / 32][W];
  const int64_t wi = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (wi >= (int64_t)*n_rows) return;  // block-uniform
  const int32_t p1 = rows[wi];
  const int32_t rs = __ldg(rstart + p1);
  const int64_t tp1 = __ldg(t + p1);
  int32_t lb[W];
  int32_t lo = rs;
#pragma unroll
  for (int k = 0; k < W; ++k) {  // nested windows: each start above the previous
    lb[k] = lower_t(t, lo, p1 + 1, tp1 - fd.d[k]);
    lo = lb[k];
  }
  // distinct counterparties of p1's windows: slots whose previous slot of
  // the same counterparty lies before the window start
  int32_t c[W];
#pragma unroll
  for (int k = 0; k < W; ++k) c[k] = 0;
  for (int32_t q = lb[0] + threadIdx.x; q <= p1; q += FAN_BATCH_BLOCK) {
    const int32_t pv = __ldg(prev + q);
#pragma unroll
    for (int k = 0; k < W; ++k) c[k] += (q >= lb[k] && pv < lb[k]) ? 1 : 0;
  }
#pragma unroll
  for (int k = 0; k < W; ++k) {
    for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
    if (lane == 0) s_c[warp][k] = c[k];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    c[k] = 0;
    for (int w = 0; w < FAN_BATCH_BLOCK / 32; ++w) c[k] += s_c[w][k];
  }
  int32_t R[W];
  int2 v[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const int32_t deg = p1 - lb[k] + 1;
    R[k] = deg - c[k];
    v[k] = make_int2(deg, c[k]);
  }
  store_df<W>(df, __ldg(eid + p1), v);
  // the row's later (new) slots
  for (int64_t p64 = p1 + 1; p64 < Ev && __ldg(rstart + p64) == rs; ++p64) {
    const int32_t p = (int32_t)p64;
    const int64_t tp = __ldg(t + p);
    const int32_t pv = __ldg(prev + p);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      int32_t l = lb[k], gone = 0;
      const int64_t tmin = tp - fd.d[k];
      while (__ldg(t + l) < tmin) {
        gone += __ldg(next + l) <= p - 1 ? 1 : 0;
        ++l;
      }
      lb[k] = l;
      R[k] += (pv >= l ? 1 : 0) - gone;
      const int32_t deg = p - l + 1;
      v[k] = make_int2(deg, deg - R[k]);
    }
    store_df<W>(df, __ldg(eid + p), v);
  }
}

template <int W>
void fan_batch_launch(const Adj& a, int64_t Ev, int64_t E, int64_t new_from,
                      const FanDeltas& fd, int2* df, cudaStream_t s) {
  const int64_t nb = E - new_from;
  if (nb <= 0 || Ev <= 0) return;
  DBuf<int32_t> rows((size_t)nb, s);
  DBuf<unsigned int> n_rows(1, s);
  AML_CUDA(cudaMemsetAsync(n_rows.p, 0, sizeof(unsigned int), s));
  AML_LAUNCH("k_batch_rows", s,
             k_batch_rows<<<grid_for(nb, 256), 256, 0, s>>>(a.pos, a.rstart, a.eid, new_from, E,
                                                            rows.p, n_rows.p));
  AML_LAUNCH("k_fan_batch", s,
             k_fan_batch<W><<<(unsigned)nb, FAN_BATCH_BLOCK, 0, s>>>(
                 a.rstart, a.t, a.eid, a.prev, a.next, Ev, fd, rows.p, n_rows.p, df));
}

}  // namespace

void fan_per_edge(const Adj& a, int64_t Ev, int64_t E, int64_t new_from, int nw,
                  const int32_t* deltas, int2* df, cudaStream_t s) {
  AML_REQUIRE(nw >= 1 && nw <= FAN_MAX_W, AML_EINTERNAL, "fan_per_edge: window count");
  if (Ev <= 0) return;
  FanDeltas fd{};
  for (int k = 0; k < nw; ++k) {
    fd.d[k] = deltas[k];
    AML_REQUIRE(k == 0 || deltas[k] <= deltas[k - 1], AML_EINTERNAL,
                "fan_per_edge: windows must be in descending order");
  }
  if (new_from > 0) {  // the new edges only
    switch (nw) {
      case 1: fan_batch_launch<1>(a, Ev, E, new_from, fd, df, s); break;
      case 2: fan_batch_launch<2>(a, Ev, E, new_from, fd, df, s); break;
      case 3: fan_batch_launch<3>(a, Ev, E, new_from, fd, df, s); break;
      default: fan_batch_launch<4>(a, Ev, E, new_from, fd, df, s); break;
    }
    return;
  }
  switch (nw) {
    case 1: fan_launch<1>(a, Ev, fd, df, s); break;
    case 2: fan_launch<2>(a, Ev, fd, df, s); break;
    case 3: fan_launch<3>(a, Ev, fd, df, s); break;
    default: fan_launch<4>(a, Ev, fd, df, s); break;
  }
}

}  // namespace aml
