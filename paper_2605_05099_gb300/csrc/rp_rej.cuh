// One-pass fill for Lemire's bounded integers when rejections are common
// (Sec. 3.2, e.g. m = 2^63 + 1, where about half the words are rejected).
// Every word is one attempt, so a thread's chunk needs no seam, and the
// bitmap kernel's second pass would only regenerate words to evaluate the
// accepted ones: with half the words rejected that doubles the engine work,
// which is what bounds this fill.  Here every word is generated once:
//   pass 1 tests each word (the low half of its product with m) and
//          compacts the accepted words of each lane through the warp's
//          staging rows into the lane's run in the CTA's parking area
//          (global memory that every tile of the CTA reuses);
//   the block scan and the look-back over tile counts give each lane its
//          first output;
//   pass 2 turns each lane's run into values (the high half of the
//          product, taken on the parked words) at its final place, the
//          whole warp on one run at a time, so every store instruction
//          writes consecutive outputs; the next run's loads are issued
//          before the current run's stores.
//
// Fragment of rp_fill_impl.cuh, included inside its namespace after the
// scans and staging helpers.

constexpr int kRejCtas = 6;   // resident CTAs per SM

template <int NT>
struct RejSmem {
  __align__(16) u64 stage[(NT / 32) * 32 * kRow];
  int wsum[32];
  int misc[8];
  u64 sh4[4];
};

// One tile.  `park` is the CTA's parking area, NT runs of C words (a lane's
// run never holds more than its C accepted values).  Returns false when the
// fill needs no further tiles (or a device check failed): the caller stops.
template <int NT, int C, class E>
__device__ bool rej_tile(const FillArgs& a, u64 k, const E& e, RejSmem<NT>& sm, u64* __restrict__ park,
                         LookbackFloor& fl) {
  static_assert(C % kStage == 0 && C <= 1024, "runs are whole staging rows; offsets fit the packed shuffle");
  constexpr int T = NT * C;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  // one reader, so that every thread takes the same branch
  if (t == 0) sm.misc[5] = ld_volatile(&a.ctrl->done_tile) < k;
  __syncthreads();
  if (sm.misc[5]) return false;
  u64* stage = sm.stage + wid * 32 * kRow;
  u64* const pw = park + (u64)wid * 32 * C;   // this warp's runs
  const u64 m = a.sp.m, thr = a.sp.thresh;
  const int half = lane >> 4, col = lane & 15;
  // ---------------- pass 1: test, compact, park
  E g = e;
  int cnt = 0;
  for (int hb = 0; hb < C / kStage; ++hb) {
    int ns = 0;
#pragma unroll
    for (int j = 0; j < kStage; j += E::kStep) {
      u64 u[E::kStep];
      g.next_step(u);
      // branch-free: every word lands in the next free slot (ns <= j <
      // kRow), which advances only for accepted words
#pragma unroll
      for (int i = 0; i < E::kStep; ++i) {
        stage[lane * kRow + ns] = u[i];
        ns += (int)(u[i] * m >= thr);
      }
    }
    __syncwarp();
    const int pk = (cnt << 5) | ns;   // run length so far and new values, one shuffle
#pragma unroll 4
    for (int r = 0; r < 32; r += 2) {
      const int rr = r + half;
      const int q = __shfl_sync(0xffffffffu, pk, rr);
      if (col < (q & 31)) pw[rr * C + (q >> 5) + col] = stage[rr * kRow + col];
    }
    __syncwarp();
    cnt += ns;
  }
  // the run was written over the whole pass and has mostly left L2 by now:
  // start bringing it back while the scan and the look-back run
  for (int i = 0; i < cnt; i += 16) asm volatile("prefetch.global.L2 [%0];" ::"l"(pw + lane * C + i));
  // ---------------- offsets
  const int off = block_exclusive_scan<NT>(cnt, sm.wsum, &sm.misc[1]);   // also orders the parked runs before pass 2
  if (t < 32) {
    unsigned long long ex = lookback_warp(a.tile_status, k, (unsigned long long)sm.misc[1], a.ctrl, fl.k, fl.inc,
                                          a.spin_max, a.stall_tile1);
    fl.k = (long long)k;
    fl.inc = ex + (unsigned long long)sm.misc[1];
    if (t == 0) {
      sm.misc[2] = (int)(ex & 0x7fffffff);
      sm.misc[3] = (int)(ex >> 31);
      sm.misc[4] = (ex == ~0ull);
    }
  }
  __syncthreads();
  if (sm.misc[4]) return false;
  const u64 base = (u64)(unsigned)sm.misc[2] | ((u64)(unsigned)sm.misc[3] << 31);
  const u64 chunk0 = k * (u64)T + (u64)t * C;
  const u64 my0 = base + (u64)off;
  if (t == NT - 1 && k + 1 == a.n_tiles && base + (u64)sm.misc[1] < a.n) {
    // ran out of tiles: report where the chain continues
    a.ctrl->total = base + (u64)sm.misc[1];
    a.ctrl->next_pos = chunk0 + (u64)C;
    a.ctrl->last_tile = k;
  }
  // the thread holding output n-1 records where the stream continues: the
  // word after its accepted word of rank n-1-my0
  if (cnt > 0 && my0 <= a.n - 1 && a.n - 1 < my0 + (u64)cnt) {
    int want = (int)(a.n - 1 - my0), p = 0;
    E h = e;
    for (; p < C; ++p) {
      const u64 u = h.next();
      if (u * m >= thr && want-- == 0) break;
    }
    a.ctrl->next_pos = chunk0 + (u64)(p + 1);
    atomicMin(&a.ctrl->done_tile, k);
  }
  // ---------------- pass 2: parked runs -> values at the output
  if (base < a.n) {
    u64* outb = (u64*)a.out + base;
    const u64 room = a.n - base;
    const int lim = room < (u64)0x7fffffff ? (int)room : 0x7fffffff;
    constexpr int Q = C / 32;   // a whole run (at most C words) in one pass of the warp
    static_assert(C % 32 == 0 && C <= 256, "a run and the next one fit the warp's registers");
    u64 v[Q];
    int o = __shfl_sync(0xffffffffu, off, 0);
    int c = min(__shfl_sync(0xffffffffu, cnt, 0), lim - o);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int i = q * 32 + lane;
      v[q] = i < c ? __ldcg(pw + i) : 0ull;
    }
    for (int r = 0; r < 32; ++r) {
      u64 w[Q];
      int o2 = 0, c2 = 0;
      if (r + 1 < 32) {
        o2 = __shfl_sync(0xffffffffu, off, r + 1);
        c2 = min(__shfl_sync(0xffffffffu, cnt, r + 1), lim - o2);
        const u64* src = pw + (r + 1) * C;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int i = q * 32 + lane;
          w[q] = i < c2 ? __ldcg(src + i) : 0ull;
        }
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int i = q * 32 + lane;
        if (i < c) outb[o + i] = __umul64hi(v[q], m);
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) v[q] = w[q];
      o = o2;
      c = c2;
    }
  }
  return true;
}

template <int NT, int C, class E>
__global__ void __launch_bounds__(NT, kRejCtas) k_rej(FillArgs a) {
  __shared__ RejSmem<NT> sm;
  E e;
  e.init_tile(a.eng, blockIdx.x, threadIdx.x, sm.sh4);
  LookbackFloor fl;
  u64* park = a.park + (u64)blockIdx.x * (u64)(NT * C);
  for (u64 k = blockIdx.x; k < a.n_tiles; k += gridDim.x) {
    if (!rej_tile<NT, C, E>(a, k, e, sm, park, fl)) break;
    e.advance(a.eng);
  }
}
