// Per-warp work loop of the persistent kernels.
//
// A warp takes `per_grab` consecutive meshlets at a time: first in fixed
// rounds (warp w of the grid's W warps takes grabs w, w + W, ...), then from
// a device work queue (one atomicAdd per grab).  Consecutive meshlets have consecutive
// payload blocks, so a grab is staged in shared memory by two bulk copies
// (`cp.async.bulk` global -> shared, issued by lane 0 and completed on an
// mbarrier): first its descriptors plus the next meshlet's (whose payload
// offset ends the range), then its whole payload range.  The meshlets are
// then handed one by one to the kernel's body.  A grab whose range does not
// look contiguous falls back to staging meshlet by meshlet.  The batch
// decoder fetches the next fixed grab's descriptors while a grab decodes.
//
// Every mbarrier wait is bounded (about a second): a wait that gives up sets
// MC_ERR_TIMEOUT in the status word and ends the warp's work; the copy it
// waited for is the only one the warp has in flight, and the warp waits for
// it once more (again bounded) before it leaves, so that the copy is unlikely
// to land in shared memory its CTA no longer owns.
#pragma once

#include "decode_warp.cuh"

namespace mcdev {

// Scratch words used by the persistent kernels.
enum { kQueue = 0, kDone = 1, kCount = 2, kViewCount = 8 };  // kViewCount..+7: per-view counts
constexpr uint32_t kMaxViews = 8;
constexpr long long kWaitCycles = 1ll << 31;  // about one second at 2 GHz

// mbarrier / bulk-copy / proxy-fence primitives (32-bit shared addresses).
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits (all lanes) for the phase with the given parity; false on every lane
// if any lane gave up after about kWaitCycles clock cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  bool ok = mbar_try_wait(bar, parity);
  if (!ok) {
    const long long t0 = clock64();
    while (!(ok = mbar_try_wait(bar, parity)) && clock64() - t0 <= kWaitCycles) {
    }
  }
  return __all_sync(kFull, ok);
}

// Shared-memory layout of the loop (bytes, per warp): the grab's descriptors
// and the next one, the mbarrier (16 bytes), then the payload blocks of a
// grab and the over-read slack, then a second descriptor buffer with its
// mbarrier (the next fixed grab's descriptors, fetched while this grab
// decodes).
__host__ __device__ inline uint32_t grab_desc_offset(uint32_t max_block_words, uint32_t per_grab) {
  return 32 * (per_grab + 1) + 16 + 4 * (per_grab * ((max_block_words + 3) & ~3u) + kSlackWords);
}
__host__ __device__ inline uint32_t grab_loop_bytes(uint32_t max_block_words, uint32_t per_grab) {
  return grab_desc_offset(max_block_words, per_grab) + 32 * (per_grab + 1) + 16;
}

// Runs the warp's share of the work queue.  Per grab, pre(m0, sdesc, cnt) is
// called by all lanes once the descriptors of the grab's cnt meshlets
// m0 .. m0 + cnt - 1 are in shared memory (sdesc, 8 words each, not yet
// validated) and returns a warp-uniform word;
// body(d, sw, j, word) is then called by all lanes for every meshlet j (batch
// index m0 + j) of the
// grab whose header passes header_ok, with sw its payload block in shared
// memory; a failed header sets MC_ERR_CORRUPT.
// After the grab's meshlets, post(m0, cnt) is called by all lanes.
struct NoPre {
  __device__ __forceinline__ uint32_t operator()(uint32_t, const uint32_t *, uint32_t) const {
    return 0;
  }
};
struct NoPost {
  __device__ __forceinline__ void operator()(uint32_t, uint32_t) const {}
};
//
// MODE 0: every grab from the queue (the ordered cull, whose grabs are taken
// in increasing order); 1: STATIC; 2: STATIC, and each fixed grab's
// descriptors are fetched into the second buffer while the grab before it
// decodes (the batch decoder; in the culls the extra state costs registers).
//
// STATIC: the first rounds take no atomic.  Warp w of the grid's W warps
// takes grabs w, w + W, w + 2W, ... for R rounds, R = 3/4 of the rounds an
// even split of the batch's grabs would need; the queue then hands out the
// grabs from R W on, which absorbs the imbalance the fixed rounds leave.
// (The atomic's cost depends on where the queue word lands in memory: with
// every grab from the queue, one 50 M-triangle batch decoded 20-40 % slower
// on some placements than on others.)
template <int MODE, class Pre, class Body, class Post = NoPost>
__device__ __forceinline__ void grab_loop(const BatchArgs &a, uint32_t per_grab, uint8_t *wbase,
                                          uint32_t lane, uint32_t *queue, uint32_t *status,
                                          Pre &&pre, Body &&body, Post &&post = Post{}) {
  constexpr bool STATIC = MODE >= 1, PREFETCH = MODE == 2;
  // descriptor buffer s (0, 1) at wbase + s * off1, its mbarrier after it
  const uint32_t off1 = grab_desc_offset(a.max_block_words, per_grab);
  const uint32_t bar0 = smem_addr(wbase + 32 * (per_grab + 1));
  uint32_t *spay = reinterpret_cast<uint32_t *>(wbase + 32 * (per_grab + 1) + 16);
  const uint32_t cap16 = (per_grab * ((a.max_block_words + 3) & ~3u)) / 4;
  const uint32_t bytes16 =
      a.payload_bytes / 16 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)(a.payload_bytes / 16);
  const uint32_t N = a.n_meshlets;
  if (lane == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + off1, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t parity = 0;          // bit s: the next phase's parity of mbarrier s
  uint32_t sel = 0;             // the buffer holding this grab's descriptors
  uint32_t m_pre = 0xFFFFFFFFu;  // the grab whose descriptors were fetched ahead
  // STATIC: this warp's next fixed grab (meshlet index), the stride between
  // its fixed grabs and the end of the fixed range
  uint32_t m_fix = 0, stride = 0, fix_end = 0;
  if (STATIC) {
    const uint32_t W = gridDim.x * (blockDim.x >> 5);
    const uint32_t G = N / per_grab + (N % per_grab ? 1u : 0u);
    fix_end = (G / W) * 3 / 4 * W * per_grab;  // <= N; N <= 2^31 leaves the sums below in range
    stride = W * per_grab;
    m_fix = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * per_grab;
  }
  for (;;) {
    uint32_t m0 = 0;
    if (STATIC && m_fix < fix_end) {
      m0 = m_fix;
      m_fix += stride;
    } else {
      if (lane == 0) m0 = atomicAdd(queue, per_grab);
      m0 = __shfl_sync(kFull, m0, 0) + fix_end;
    }
    if (m0 >= N) break;
    const uint32_t cnt = min(per_grab, N - m0);
    const uint32_t nd = cnt + (m0 + cnt < N ? 1u : 0u);
    fence_proxy_async();  // the previous grab's shared-memory accesses before the async writes
    __syncwarp();
    const uint32_t *sdesc = reinterpret_cast<const uint32_t *>(wbase + sel * off1);
    const uint32_t bar = bar0 + sel * off1;
    if (!(PREFETCH && m0 == m_pre) && lane == 0) {  // not fetched ahead: fetch now
      mbar_expect_tx(bar, 32 * nd);
      bulk_g2s(smem_addr(sdesc), a.desc + m0, 32 * nd, bar);
    }
    if (!mbar_wait(bar, (parity >> sel) & 1u)) {
      if (lane == 0) set_status(status, MC_ERR_TIMEOUT);
      mbar_wait(bar, (parity >> sel) & 1u);  // a second bounded wait for the copy in flight
      return;
    }
    parity ^= 1u << sel;
    const uint32_t start16 = sdesc[0];
    const uint32_t end16 = m0 + cnt < N ? sdesc[8 * cnt] : bytes16;
    bool staged = end16 >= start16 && end16 - start16 <= cap16 && end16 <= bytes16;
    if (staged && end16 > start16) {
      if (lane == 0) {
        mbar_expect_tx(bar, 16 * (end16 - start16));
        bulk_g2s(smem_addr(spay), a.payload + 16ull * start16, 16 * (end16 - start16), bar);
      }
      if (!mbar_wait(bar, (parity >> sel) & 1u)) {
        if (lane == 0) set_status(status, MC_ERR_TIMEOUT);
        mbar_wait(bar, (parity >> sel) & 1u);  // a second bounded wait for the copy in flight
        return;
      }
      parity ^= 1u << sel;
    }
    // the next fixed grab's descriptors into the other buffer, while this
    // grab decodes (the warp takes that grab next, so none is left in flight)
    m_pre = 0xFFFFFFFFu;
    if (PREFETCH && m_fix < fix_end) {
      const uint32_t cn = min(per_grab, N - m_fix);
      const uint32_t ndn = cn + (m_fix + cn < N ? 1u : 0u);
      if (lane == 0) {
        mbar_expect_tx(bar0 + (sel ^ 1u) * off1, 32 * ndn);
        bulk_g2s(smem_addr(wbase + (sel ^ 1u) * off1), a.desc + m_fix, 32 * ndn,
                 bar0 + (sel ^ 1u) * off1);
      }
      m_pre = m_fix;
    }
    const uint32_t word = pre(m0, sdesc, cnt);
    // the grab's header checks and staged ranges, one lane per meshlet
    bool ok_l = false, in_l = false;
    if (lane < cnt) {
      const uint4 *sd = reinterpret_cast<const uint4 *>(sdesc) + 2 * lane;
      const Desc d = with_attrs(unpack_desc(sd[0], sd[1]), a);
      ok_l = header_ok(d, a);
      const uint32_t padded16 = ((block_words(d) + 3) & ~3u) / 4;
      in_l = d.off16 >= start16 && d.off16 - start16 + padded16 <= end16 - start16;
    }
    const uint32_t ok_mask = __ballot_sync(kFull, ok_l), in_mask = __ballot_sync(kFull, in_l);
    for (uint32_t j = 0; j < cnt; j++) {
      const uint4 *sd = reinterpret_cast<const uint4 *>(sdesc) + 2 * j;
      const Desc d = with_attrs(unpack_desc(sd[0], sd[1]), a);
      if (!((ok_mask >> j) & 1u)) {
        if (lane == 0) set_status(status, MC_ERR_CORRUPT);
        continue;
      }
      const uint32_t *sw;
      if (staged && ((in_mask >> j) & 1u)) {
        sw = spay + 4 * (d.off16 - start16);
      } else {
        staged = false;  // spay is reused meshlet by meshlet from here on
        __syncwarp();
        stage_payload(d, a.payload, spay, lane);
        __syncwarp();
        sw = spay;
      }
      body(d, sw, j, word, m0 + j);
    }
    __syncwarp();
    post(m0, cnt);
    if (PREFETCH && m_pre != 0xFFFFFFFFu) sel ^= 1u;
  }
}

// The work loop with two meshlets per warp (per_grab >= 2): grabs are taken
// and staged as in grab_loop (the same steps, written out here so that each
// loop keeps its own registers), and the meshlets of a grab are handed out
// in pairs, meshlet j + h to the half h = lane / 16: body(d, live, sw, m) is
// called by all lanes with this half's descriptor, whether it holds a
// meshlet that passed header_ok (live), its staged block sw and its batch
// index m.  Blocks outside the grab's staged range are staged pair by pair
// into the first two slots of the payload buffer.
template <class Body>
__device__ __forceinline__ void grab_loop_pairs(const BatchArgs &a, uint32_t per_grab,
                                                uint8_t *wbase, uint32_t lane, uint32_t *queue,
                                                uint32_t *status, Body &&body) {
  const uint32_t *sdesc = reinterpret_cast<const uint32_t *>(wbase);
  const uint32_t bar = smem_addr(wbase + 32 * (per_grab + 1));
  uint32_t *spay = reinterpret_cast<uint32_t *>(wbase + 32 * (per_grab + 1) + 16);
  const uint32_t slot_words = (a.max_block_words + 3) & ~3u;
  const uint32_t cap16 = (per_grab * slot_words) / 4;
  const uint32_t bytes16 =
      a.payload_bytes / 16 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)(a.payload_bytes / 16);
  const uint32_t N = a.n_meshlets;
  const uint32_t h = lane >> 4, hl = lane & 15u;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  uint32_t parity = 0;
  for (;;) {
    uint32_t m0 = 0;
    if (lane == 0) m0 = atomicAdd(queue, per_grab);
    m0 = __shfl_sync(kFull, m0, 0);
    if (m0 >= N) break;
    const uint32_t cnt = min(per_grab, N - m0);
    const uint32_t nd = cnt + (m0 + cnt < N ? 1u : 0u);
    fence_proxy_async();  // the previous grab's shared-memory accesses before the async writes
    __syncwarp();
    if (lane == 0) {
      mbar_expect_tx(bar, 32 * nd);
      bulk_g2s(smem_addr(wbase), a.desc + m0, 32 * nd, bar);
    }
    if (!mbar_wait(bar, parity)) {
      if (lane == 0) set_status(status, MC_ERR_TIMEOUT);
      mbar_wait(bar, parity);  // a second bounded wait for the copy in flight
      return;
    }
    parity ^= 1u;
    const uint32_t start16 = sdesc[0];
    const uint32_t end16 = m0 + cnt < N ? sdesc[8 * cnt] : bytes16;
    bool staged = end16 >= start16 && end16 - start16 <= cap16 && end16 <= bytes16;
    if (staged && end16 > start16) {
      if (lane == 0) {
        mbar_expect_tx(bar, 16 * (end16 - start16));
        bulk_g2s(smem_addr(spay), a.payload + 16ull * start16, 16 * (end16 - start16), bar);
      }
      if (!mbar_wait(bar, parity)) {
        if (lane == 0) set_status(status, MC_ERR_TIMEOUT);
        mbar_wait(bar, parity);  // a second bounded wait for the copy in flight
        return;
      }
      parity ^= 1u;
    }
    for (uint32_t j = 0; j < cnt; j += 2) {
      const uint32_t jj = j + h;
      Desc d{};
      bool live = jj < cnt;
      if (live) {
        const uint4 *sd = reinterpret_cast<const uint4 *>(sdesc) + 2 * jj;
        d = with_attrs(unpack_desc(sd[0], sd[1]), a);
        live = header_ok(d, a);
        if (!live && hl == 0) set_status(status, MC_ERR_CORRUPT);
        if (!live) d = Desc{};  // an idle half decodes nothing
      }
      const uint32_t *sw = spay;
      bool in_range = true;
      if (live) {
        const uint32_t padded16 = ((block_words(d) + 3) & ~3u) / 4;
        in_range = staged && d.off16 >= start16 && d.off16 - start16 + padded16 <= end16 - start16;
        if (in_range) sw = spay + 4 * (d.off16 - start16);
      }
      if (__any_sync(kFull, !in_range)) {  // this pair's blocks, each into its own slot
        staged = false;  // spay is reused pair by pair from here on
        __syncwarp();
        uint32_t *dst = spay + h * slot_words;
        if (live) {
          const uint4 *src = reinterpret_cast<const uint4 *>(a.payload) + d.off16;
          const uint32_t n4 = (block_words(d) + 3) >> 2;
          for (uint32_t i = hl; i < n4; i += 16) reinterpret_cast<uint4 *>(dst)[i] = __ldg(src + i);
        }
        __syncwarp();
        sw = dst;
      }
      body(d, live, sw, m0 + jj);
    }
    __syncwarp();
  }
}

}  // namespace mcdev
