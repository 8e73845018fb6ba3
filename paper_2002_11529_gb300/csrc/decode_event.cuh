// Per-event UT raw-bank decoding (Sec. IV, Table I of the paper) as a
// device function, shared by the single-pass decode kernel and the
// persistent batched kernel.
//
// One block decodes one event: a bulk (TMA) copy stages the event's raw
// words in shared memory, one thread per bank checks the directory and
// header and counts hits, a block scan gives the event-local offsets, a
// decoupled look-back over the previous events gives the global hit base,
// and one thread per hit writes the decoded SoA at its (optionally
// half-strip-ranked) slot.  Banks of more than kSmallBank hits are ranked
// by a warp counting sort.
#pragma once

#include "common.cuh"

namespace utc {

constexpr int kMaxDecodeThreads = 1024;
constexpr int kSmallBank = 64;          // banks up to this size rank by direct counting
constexpr int kBigWarps = 1;            // warps that sort larger banks
constexpr int kKeyBins = 1024;          // half-strip keys (strips <= 512)
constexpr uint32_t kStageWordsDefault = 8192;
constexpr uint32_t kMapCapDefault = 8192;
// Bank-order decode: a smaller stage and bank map (36 KB of shared memory
// per 256-thread block with 4 x 256 sectors, six blocks per SM instead of
// four) measured faster on events of 500-15000 hits; larger events take the
// global-memory and map-free paths.
constexpr uint32_t kStageWordsBank = 6144;
constexpr uint32_t kMapCapBank = 4096;

// Tile (event) state of the look-back, 64-bit: flag in bits 62-63.
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

struct DecodeArgs {
    const uint32_t* raw;
    uint64_t n_words;
    const uint64_t* ev_off;
    int n_events;
    int S;
    float* x;
    float* z;
    uint16_t* sector;
    uint8_t* layer;
    uint32_t* id;
    uint32_t* hit_off;
    uint32_t capacity;
    float x_min, sector_pitch, half_pitch;
    int strips;
    float zl[4];
    unsigned int* ticket;
    unsigned long long* tile_state;
    unsigned long long* status;
    uint32_t stage_words;
    uint32_t map_cap;            // events up to this many hits use the mapped, vector-store path
    int vec_ok;                  // output arrays are 16-byte aligned
    long long spin_limit;        // polls of a bounded wait before UT_ERR_TIMEOUT
};

// All five output arrays start on a 16-byte boundary (vector stores allowed).
inline int hits_aligned16(const ut_hits* h) {
    const uintptr_t m = (uintptr_t)h->x | (uintptr_t)h->z | (uintptr_t)h->sector | (uintptr_t)h->layer |
                        (uintptr_t)h->id;
    return (m & 15u) == 0;
}

struct HitOut {
    float* x;
    float* z;
    uint16_t* sector;
    uint8_t* layer;
    uint32_t* id;
};

// Layer l and sector s of bank b = l * S + s, by comparison (no division).
__device__ __forceinline__ void bank_ls(int b, int S, int& l, int& s) {
    l = (int)(b >= S) + (int)(b >= 2 * S) + (int)(b >= 3 * S);
    s = b - l * S;
}

// x at y = 0 of hit word w in sector s (Sec. IV): x0_s + (h + 1/2) pitch/2,
// x0_s = s * sector_pitch + x_min.  Each float operation is a separate IEEE
// op (no contraction: -fmad=false).
__device__ __forceinline__ float decode_x(const DecodeArgs& a, int s, uint32_t w) {
    const uint32_t h = half_strip(w);
    const float x0 = __fadd_rn(__fmul_rn((float)s, a.sector_pitch), a.x_min);
    const float c = __fmul_rn(__fadd_rn((float)h, 0.5f), a.half_pitch);
    return __fadd_rn(x0, c);
}

__device__ __forceinline__ void write_hit(const DecodeArgs& a, uint32_t o, int l, int s, uint32_t w, float* sx,
                                          uint32_t sx_cap, uint32_t local) {
    if (!chk(o < a.capacity, a.status, 101)) return;
    const float x = decode_x(a, s, w);
    a.x[o] = x;
    if (sx != nullptr && local < sx_cap) sx[local] = x;
    a.z[o] = a.zl[l];
    a.sector[o] = (uint16_t)s;
    a.layer[o] = (uint8_t)l;
    a.id[o] = ((uint32_t)l << 24) | ((uint32_t)s << 16) | w;
}

// Block-wide exclusive scan of cnt[0..n) in place, cnt[n] = total; returns
// the total.  n may exceed the block size (each thread scans a contiguous
// run).  Ends with a barrier: every thread may read cnt[0..n] on return.
static __device__ uint32_t block_exclusive_scan(uint32_t* cnt, int n, uint32_t* warp_tot) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    const int b0 = min(tid * per, n), b1 = min(b0 + per, n);
    uint32_t local = 0;
    for (int b = b0; b < b1; ++b) local += cnt[b];
    // warp inclusive scan of the per-thread sums
    const int lane = tid & 31, wid = tid >> 5;
    uint32_t v = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = nt >> 5;
        uint32_t w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += t;
        }
        if (lane < nw) warp_tot[lane] = w;  // inclusive per warp
    }
    __syncthreads();
    uint32_t run = (v - local) + (wid > 0 ? warp_tot[wid - 1] : 0u);
    const uint32_t total = warp_tot[(nt >> 5) - 1];
    for (int b = b0; b < b1; ++b) {
        const uint32_t c = cnt[b];
        cnt[b] = run;
        run += c;
    }
    if (tid == 0) cnt[n] = total;
    __syncthreads();
    return total;
}

// Decoupled look-back (single-pass prefix sum across events): returns the
// sum of the aggregates of all events before `e`.  Executed by one warp;
// each step reads the states of 128 predecessors (four per lane, lane-major
// by distance) and waits only for those nearer than the nearest inclusive
// prefix.
static __device__ unsigned long long lookback(unsigned long long* tile_state, int e, unsigned long long* status,
                                              long long spin_limit) {
    const int lane = threadIdx.x & 31;
    unsigned long long excl = 0;
    int j = e - 1;  // nearest predecessor not yet summed
    long long spins = 0;
    while (j >= 0) {
        unsigned long long st[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int idx = j - (lane * 4 + t);
            st[t] = idx >= 0 ? ld_volatile_u64(tile_state + idx) : kFlagPrefix;
        }
        int tp;
        uint32_t pmask;
        int stop;
        for (;;) {
            tp = 4;
#pragma unroll
            for (int t = 3; t >= 0; --t)
                if ((st[t] >> 62) == 2) tp = t;
            pmask = __ballot_sync(0xffffffffu, tp < 4);
            stop = pmask ? __ffs(pmask) - 1 : 32;  // lane holding the nearest prefix
            bool missing = false;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool needed = lane < stop || (lane == stop && t < tp);
                missing |= needed && (st[t] >> 62) == 0;
            }
            if (!__any_sync(0xffffffffu, missing)) break;
            if (++spins > spin_limit) {
                if (lane == 0) report(status, UT_ERR_TIMEOUT, e, -1);
                return excl;
            }
            __nanosleep(32);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int idx = j - (lane * 4 + t);
                if (idx >= 0 && (st[t] >> 62) == 0) st[t] = ld_volatile_u64(tile_state + idx);
            }
        }
        unsigned long long v = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (lane < stop || (lane == stop && t <= tp)) v += st[t] & kValueMask;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        excl += v;
        if (pmask) break;
        j -= 128;
    }
    return excl;
}

// Stable rank of key[k] among key[0..n) (small banks): number of keys that
// are smaller, or equal and earlier.
__device__ __forceinline__ uint32_t rank_small(const uint16_t* w16, uint32_t n, uint32_t k, uint32_t hk) {
    uint32_t r = 0;
    for (uint32_t j = 0; j < n; ++j) {
        const uint32_t hj = min(half_strip(w16[j]), (uint32_t)(kKeyBins - 1));
        r += (hj < hk) || (hj == hk && j < k);
    }
    return r;
}

// Shared memory used by decode_event.
struct DecodeSmem {
    uint32_t* bigcnt;            // kBigWarps * kKeyBins (SORT only)
    uint32_t* off;               // B + 1: event-local exclusive offsets, off[B] = total
    uint32_t* stage;             // stage_words, 16-byte aligned
    uint64_t* mbar;              // bulk-copy barrier (initialised by the caller)
    unsigned long long* s_base;  // global hit base of the event
    uint32_t* warp_tot;          // kMaxDecodeThreads / 32
    uint16_t* bmap;              // map_cap: bank of each hit (null: mapped path off)
    uint16_t* srcmap;            // map_cap: hit written at each output position
    uint16_t* list16;            // kMapList: banks of 9..kNetBank hits (null: sorted where met)
    uint16_t* listw;             // kMapList: banks of kNetBank+1..kSmallBank hits
    int* nlist;                  // 2 counters of the lists
};

// Capacity of each of the two bank lists of the sorted maps.
constexpr int kMapList = 256;

__device__ __forceinline__ const uint16_t* bank_words(const uint32_t* evw, int b) {
    return reinterpret_cast<const uint16_t*>(evw + evw[b] + 1);
}

// Ranks the hits of banks of more than kSmallBank hits by a counting sort
// on the half-strip key, one warp per bank (histogram, exclusive scan of the
// bins, then a stable pass in word order where equal keys inside a 32-word
// chunk are ranked with a match mask).  place(b, pos, k, w): word k of bank
// b goes to position pos of the bank.
template <class Place>
__device__ void rank_big_banks(const uint32_t* off, int B, const uint32_t* evw, uint32_t* bigcnt, Place place) {
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    if (wid >= kBigWarps) return;
    uint32_t* cnt = bigcnt + wid * kKeyBins;
    for (int b0 = wid * 32; b0 < B; b0 += kBigWarps * 32) {
        const int bl = b0 + lane;
        const bool big = bl < B && (off[bl + 1] - off[bl]) > (uint32_t)kSmallBank;
        uint32_t mask = __ballot_sync(0xffffffffu, big);
        while (mask) {
            const int b = b0 + __ffs(mask) - 1;
            mask &= mask - 1;
            const uint32_t n = off[b + 1] - off[b];
            const uint16_t* w16 = bank_words(evw, b);
            for (int q = lane; q < kKeyBins; q += 32) cnt[q] = 0;
            __syncwarp();
            for (uint32_t k = lane; k < n; k += 32)
                atomicAdd(&cnt[min(half_strip(w16[k]), (uint32_t)(kKeyBins - 1))], 1u);
            __syncwarp();
            uint32_t run = 0;
            for (int q = 0; q < kKeyBins / 32; ++q) run += cnt[lane * (kKeyBins / 32) + q];
            uint32_t incl = run;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += t;
            }
            uint32_t acc = incl - run;
            for (int q = 0; q < kKeyBins / 32; ++q) {
                const uint32_t c = cnt[lane * (kKeyBins / 32) + q];
                cnt[lane * (kKeyBins / 32) + q] = acc;
                acc += c;
            }
            __syncwarp();
            for (uint32_t k0 = 0; k0 < n; k0 += 32) {
                const uint32_t k = k0 + lane;
                const bool valid = k < n;
                const uint32_t w = valid ? w16[k] : 0u;
                const uint32_t hk = valid ? min(half_strip(w), (uint32_t)(kKeyBins - 1)) : kKeyBins + lane;
                const uint32_t peers = __match_any_sync(0xffffffffu, hk);
                const uint32_t before = __popc(peers & lanemask_lt());
                const uint32_t pos = valid ? cnt[hk] + before : 0u;
                __syncwarp();
                if (valid && before == 0) cnt[hk] += __popc(peers);
                __syncwarp();
                if (valid) place(b, pos, k, w);
            }
            __syncwarp();
        }
    }
}

// Decoded hit of output position o (event-local) whose word is w in bank b.
struct DecodedHit {
    float x, z;
    uint32_t s, l, id;
};

__device__ __forceinline__ DecodedHit decoded_hit(const DecodeArgs& a, int b, uint32_t w) {
    int l, s;
    bank_ls(b, a.S, l, s);
    DecodedHit h;
    h.x = decode_x(a, s, w);
    h.z = a.zl[l];
    h.s = (uint32_t)s;
    h.l = (uint32_t)l;
    h.id = ((uint32_t)l << 24) | ((uint32_t)s << 16) | w;
    return h;
}

// Bitonic sorting network on N keys held in registers (N a power of two;
// every index is a compile-time constant, so nothing leaves the registers).
template <int N>
__device__ __forceinline__ void sort_network(uint32_t (&k)[N]) {
#pragma unroll
    for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t x = k[i], y = k[l];
                    const uint32_t lo = min(x, y), hi = max(x, y);
                    const bool up = (i & kk) == 0;
                    k[i] = up ? lo : hi;
                    k[l] = up ? hi : lo;
                }
            }
        }
    }
}

// A bank of n <= N hits sorted by one thread: keys (half-strip << 6 | word
// index, unique, so the order is the stable one) sorted in registers, then
// the word position of each output slot written to srcm and the bank to
// bmap.
template <int N>
__device__ __forceinline__ void sort_small_bank(const uint16_t* w16, uint32_t wpos0, uint32_t n, int b, uint32_t j0,
                                                uint16_t* bmap, uint16_t* srcm) {
    uint32_t k[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
        k[i] = (uint32_t)i < n ? ((min(half_strip(w16[i]), (uint32_t)(kKeyBins - 1)) << 6) | (uint32_t)i) : 0xFFFFFFFFu;
    sort_network<N>(k);
#pragma unroll
    for (int r = 0; r < N; ++r) {
        if ((uint32_t)r < n) {
            srcm[j0 + r] = (uint16_t)(wpos0 + (k[r] & 63u));
            bmap[j0 + r] = (uint16_t)b;
        }
    }
}

// Banks of at most this many hits are sorted by their own thread (sorting
// network of 8 or 16 keys); larger ones up to kSmallBank by the whole warp
// that meets them.
constexpr int kNetBank = 16;

// Sorts one bank of kNetBank < n <= kSmallBank hits with the L lanes of a
// warp (mask wmask, lanes 0..L-1): the keys (half-strip << 6) | word index
// are written to the bank's own range of srcm, each lane counts the keys
// below those of its words (rank; the keys are unique, so the order is the
// stable one), and after the warp has read every key the word position of
// each hit is stored at its rank.
__device__ __forceinline__ void warp_sort_bank(const uint16_t* w16, uint32_t wpos0, uint32_t n, int b, uint32_t j0,
                                               uint16_t* bmap, uint16_t* srcm, int lane, int L, uint32_t wmask) {
    uint16_t* K = srcm + j0;
    for (uint32_t j = (uint32_t)lane; j < n; j += (uint32_t)L) {
        K[j] = (uint16_t)((min(half_strip(w16[j]), (uint32_t)(kKeyBins - 1)) << 6) | j);
        bmap[j0 + j] = (uint16_t)b;
    }
    __syncwarp(wmask);
    if (n <= (uint32_t)L) {  // one word per lane
        const uint32_t j = (uint32_t)lane;
        const uint32_t key = j < n ? (uint32_t)K[j] : 0u;
        uint32_t r = 0;
        for (uint32_t i = 0; i < n; ++i) r += (uint32_t)((uint32_t)K[i] < key);
        __syncwarp(wmask);
        if (j < n) K[r] = (uint16_t)(wpos0 + j);
        __syncwarp(wmask);
        return;
    }
    // three words per lane in each round
    for (uint32_t jb = 0; jb < n; jb += 3u * (uint32_t)L) {
        uint32_t key[3], r[3] = {0u, 0u, 0u};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const uint32_t j = jb + (uint32_t)lane + (uint32_t)(m * L);
            key[m] = j < n ? (uint32_t)K[j] : 0u;
        }
        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t ki = K[i];
#pragma unroll
            for (int m = 0; m < 3; ++m) r[m] += (uint32_t)(ki < key[m]);
        }
        __syncwarp(wmask);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const uint32_t j = jb + (uint32_t)lane + (uint32_t)(m * L);
            if (j < n) K[r[m]] = (uint16_t)(wpos0 + j);
        }
        __syncwarp(wmask);
    }
}

// Shared-memory maps of an event of at most map_cap hits, built before its
// global base is known.  bmap[i] = bank of output position i.  SORT:
// srcmap[i] = position, in the event's 16-bit words, of the word at output
// position i.  One thread per bank: a bank of at most 8 hits is sorted at
// once by a sorting network in registers.  With the block's bank lists
// (sm.list16, sm.listw), banks of 9..kNetBank hits and of up to kSmallBank
// hits are listed, and after a barrier sorted by networks of 16 keys one
// per thread and by whole warps (warp_sort_bank), spread over all warps;
// without them (or when a list is full) they are sorted by the thread, or
// the warp, that meets them.  Larger banks (any_big: the event has some)
// are ranked by rank_big_banks straight into srcmap.  The maps are complete
// after the next __syncthreads of the caller.
template <bool SORT>
__device__ void map_event(const DecodeArgs& a, const DecodeSmem& sm, const uint32_t* evw, bool any_big,
                          uint64_t nw) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int B = 4 * a.S;
    const uint32_t* off = sm.off;
    uint16_t* bmap = sm.bmap;
    uint16_t* srcm = sm.srcmap;
    const int lane = tid & 31, wt0 = tid - lane;
    const int L = min(32, nt - wt0);  // lanes of this warp
    const uint32_t wmask = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
    const bool lists = SORT && sm.list16 != nullptr;
    const uint16_t* w16 = reinterpret_cast<const uint16_t*>(evw);
    // the same number of rounds for every lane of a warp (warp-wide sorts)
    for (int k0 = 0; wt0 + k0 < B; k0 += nt) {
        const int b = tid + k0;
        bool coop = false;
        if (b < B) {
            const uint32_t j0 = off[b], n = off[b + 1] - j0;
            if (chk(j0 + n <= a.map_cap, a.status, 104)) {
                if (SORT && n <= (uint32_t)kSmallBank) {
                    if (chk((uint64_t)evw[b] + 1 + (n + 1) / 2 <= nw, a.status, 110)) {
                        const uint32_t wpos0 = 2u * (evw[b] + 1u);
                        if (n <= 8) {
                            sort_small_bank<8>(w16 + wpos0, wpos0, n, b, j0, bmap, srcm);
                        } else if (n <= (uint32_t)kNetBank) {
                            const int idx = lists ? atomicAdd(&sm.nlist[0], 1) : kMapList;
                            if (idx < kMapList) sm.list16[idx] = (uint16_t)b;
                            else sort_small_bank<kNetBank>(w16 + wpos0, wpos0, n, b, j0, bmap, srcm);
                        } else {
                            const int idx = lists ? atomicAdd(&sm.nlist[1], 1) : kMapList;
                            if (idx < kMapList) sm.listw[idx] = (uint16_t)b;
                            else coop = true;
                        }
                    }
                } else {
                    for (uint32_t j = j0; j < j0 + n; ++j) bmap[j] = (uint16_t)b;
                }
            }
        }
        if constexpr (SORT) {
            uint32_t cm = __ballot_sync(wmask, coop);
            while (cm) {
                const int src = __ffs(cm) - 1;
                cm &= cm - 1;
                const int bb = wt0 + k0 + src;
                const uint32_t j0 = off[bb], n = off[bb + 1] - j0;
                const uint32_t wpos0 = 2u * (evw[bb] + 1u);
                warp_sort_bank(w16 + wpos0, wpos0, n, bb, j0, bmap, srcm, lane, L, wmask);
            }
        }
    }
    if constexpr (SORT) {
        if (lists) {
            // The listed banks, spread over all warps: the hot sectors are
            // neighbours, and sorted where met they would fall to one or
            // two warps.  Banks of 9..kNetBank hits: one per thread, entry
            // lane * warps + warp (so each warp takes some); larger ones: one
            // per warp at a time.
            __syncthreads();
            const int n16 = min(sm.nlist[0], kMapList), nwl = min(sm.nlist[1], kMapList);
            const int nwarps = (nt + 31) >> 5, w = tid >> 5;
            const int slot = (nt & 31) == 0 ? lane * nwarps + w : tid;
            for (int i = slot; i < n16; i += nt) {
                const int b = sm.list16[i];
                const uint32_t j0 = off[b], n = off[b + 1] - j0;
                const uint32_t wpos0 = 2u * (evw[b] + 1u);
                sort_small_bank<kNetBank>(w16 + wpos0, wpos0, n, b, j0, bmap, srcm);
            }
            for (int i = w; i < nwl; i += nwarps) {
                const int b = sm.listw[i];
                const uint32_t j0 = off[b], n = off[b + 1] - j0;
                const uint32_t wpos0 = 2u * (evw[b] + 1u);
                warp_sort_bank(w16 + wpos0, wpos0, n, b, j0, bmap, srcm, lane, L, wmask);
            }
        }
        if (any_big)
            rank_big_banks(off, B, evw, sm.bigcnt, [&](int b, uint32_t pos, uint32_t k, uint32_t) {
                srcm[off[b] + pos] = (uint16_t)(2u * (evw[b] + 1u) + k);
            });
    }
}

// Writes of an event in output order; groups of four outputs that start on
// a 16-byte boundary in global memory use vector stores.  SORT: the bank and
// the source word of each output position come from the shared-memory maps.
// Bank order: output position o is word o - off[b] of the bank b holding it,
// read from the bank map when the event has one (from_map), else found by a
// binary search over the event-local offsets for the first output of a
// group and by a forward walk for the others.
template <bool SORT>
__device__ void write_mapped(const DecodeArgs& a, int e, const DecodeSmem& sm, const uint32_t* evw,
                             unsigned long long base, uint32_t total, bool fits, float* sx, uint32_t sx_cap,
                             uint64_t nw, bool from_map) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int B = 4 * a.S;
    const uint32_t* off = sm.off;
    const uint16_t* bmap = sm.bmap;
    const uint16_t* srcm = sm.srcmap;
    // bank of output position o: from the map (SORT) or from the offsets,
    // starting at bank `hint` (a bank at or before it)
    auto bank_of = [&](uint32_t o, int hint) -> int {
        if constexpr (SORT) {
            return (int)ld_chk(bmap, o, a.map_cap, a.status, 107);
        } else {
            if (from_map) return (int)ld_chk(bmap, o, a.map_cap, a.status, 107);
            int b = hint;
            while (off[b + 1] <= o) ++b;
            return b;
        }
    };
    auto hit_at = [&](uint32_t o, int b) -> DecodedHit {
        const long long wpos = SORT ? (long long)ld_chk(srcm, o, a.map_cap, a.status, 107)
                                    : 2ll * ((long long)evw[b] + 1) + (long long)(o - off[b]);
        const uint32_t w = (uint32_t)ld_chk(reinterpret_cast<const uint16_t*>(evw), wpos, 2ll * (long long)nw,
                                            a.status, 106);
        if ((w & 0x3FFu) >= (uint32_t)a.strips) report(a.status, UT_ERR_STRIP, e, b);
        return decoded_hit(a, b, w);
    };
    auto one = [&](uint32_t o) {
        const int b = bank_of(o, SORT || from_map ? 0 : find_bank(off, B, o));
        const DecodedHit h = hit_at(o, b);
        if (sx != nullptr && o < sx_cap) sx[o] = h.x;
        if (!fits) return;
        const size_t g = (size_t)(base + o);
        if (!chk(g < a.capacity, a.status, 102)) return;
        a.x[g] = h.x;
        a.z[g] = h.z;
        a.sector[g] = (uint16_t)h.s;
        a.layer[g] = (uint8_t)h.l;
        a.id[g] = h.id;
    };
    uint32_t head = a.vec_ok ? (uint32_t)((4u - (uint32_t)(base & 3u)) & 3u) : total;
    if (head > total) head = total;
    const uint32_t nq = (total - head) / 4;
    for (uint32_t o = tid; o < head; o += nt) one(o);
    for (uint32_t q = tid; q < nq; q += nt) {
        const uint32_t o = head + 4 * q;
        DecodedHit h[4];
        int b = SORT || from_map ? 0 : find_bank(off, B, o);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            b = bank_of(o + j, b);
            h[j] = hit_at(o + j, b);
            if (sx != nullptr && o + j < sx_cap) sx[o + j] = h[j].x;
        }
        if (!fits) continue;
        const size_t g = (size_t)(base + o);
        if (!chk(g + 4 <= a.capacity, a.status, 103)) continue;
        *reinterpret_cast<float4*>(a.x + g) = make_float4(h[0].x, h[1].x, h[2].x, h[3].x);
        *reinterpret_cast<float4*>(a.z + g) = make_float4(h[0].z, h[1].z, h[2].z, h[3].z);
        *reinterpret_cast<uint2*>(a.sector + g) = make_uint2(h[0].s | (h[1].s << 16), h[2].s | (h[3].s << 16));
        *reinterpret_cast<uint32_t*>(a.layer + g) = h[0].l | (h[1].l << 8) | (h[2].l << 16) | (h[3].l << 24);
        *reinterpret_cast<uint4*>(a.id + g) = make_uint4(h[0].id, h[1].id, h[2].id, h[3].id);
    }
    for (uint32_t o = head + 4 * nq + tid; o < total; o += nt) one(o);
}

// Decode event e with the whole block.  `phase` is the parity of the bulk
// copy barrier's next phase (toggled when a copy completes); `tma_ok` turns
// false (for the whole block) after a copy that did not complete within two
// wait limits: the stage region may still receive it, so the caller stops
// using shared memory that overlaps the stage (it waits once more, bounded,
// before it exits).  sx (nullable)
// receives the event-local decoded x of positions < sx_cap.  On return
// (after a __syncthreads by the caller) sm.off holds the event-local
// offsets and *sm.s_base the event's global base.
template <bool SORT>
__device__ void decode_event(const DecodeArgs& a, int e, const DecodeSmem& sm, uint32_t& phase, bool& tma_ok,
                             float* sx, uint32_t sx_cap) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int S = a.S, B = 4 * S;
    uint32_t* off = sm.off;
    uint32_t* stage = sm.stage;
    const uint64_t ws = a.ev_off[e], we = a.ev_off[e + 1];
    const bool ev_ok = we >= ws && we <= a.n_words && (we - ws) >= (uint64_t)B;
    const uint64_t nw = ev_ok ? we - ws : 0;
    const uint32_t* evw = a.raw + (ev_ok ? ws : 0);

    if (SORT && sm.nlist != nullptr && tid == 0) sm.nlist[0] = sm.nlist[1] = 0;  // read after the scan's barriers

    // Stage the whole event (16-byte aligned superset) with one bulk copy.
    // After a copy that did not complete in time the block stops using the
    // stage (tma_ok = false) and reads raw words from global memory.
    if (ev_ok) {
        const uint64_t al0 = ws & ~3ull, al1 = (we + 3) & ~3ull;
        const uint64_t words = al1 - al0;
        if (tma_ok && words <= a.stage_words) {
            if (tid == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(sm.mbar, (uint32_t)(words * 4));
                const uint32_t* src = a.raw + al0;
                uint64_t done = 0;
                while (done < words) {
                    const uint32_t chunk = (uint32_t)((words - done) < 8192ull ? (words - done) : 8192ull);  // 32 KB
                    bulk_copy_g2s(stage + done, src + done, chunk * 4, sm.mbar);
                    done += chunk;
                }
            }
            // the outcome is made the same for the whole block
            if (__syncthreads_and(mbar_wait_bounded(sm.mbar, phase, a.spin_limit))) {
                evw = stage + (ws - al0);
                phase ^= 1u;
            } else {
                // the copy did not complete in time: record it, read this
                // event from global memory, and wait (bounded) once more so
                // that the copy cannot land later in shared memory the block
                // reuses; if it is still in flight the block stops using the
                // stage region (tma_ok = false: the caller ends its work)
                if (tid == 0) report(a.status, UT_ERR_TIMEOUT, e, -1);
                if (__syncthreads_and(mbar_wait_bounded(sm.mbar, phase, a.spin_limit))) phase ^= 1u;
                else tma_ok = false;
            }
        }
    } else if (tid == 0) {
        report(a.status, UT_ERR_DIR, e, 0);
    }

    // Hit counting with directory / header checks (one thread per bank).
    bool big = false;  // a bank of more than kSmallBank hits (ranked by rank_big_banks)
    for (int b = tid; b < B; b += nt) {
        uint32_t n = 0;
        if (ev_ok) {
            const uint32_t d = evw[b];
            if ((uint64_t)d >= (uint64_t)B && (uint64_t)d + 1 <= nw) {
                const uint32_t hdr = evw[d];
                const uint32_t nn = hdr & 0xFFFFu;
                if ((uint64_t)d + 1 + (nn + 1) / 2 > nw) {
                    report(a.status, UT_ERR_DIR, e, b);
                } else if ((hdr >> 16) != (uint32_t)b) {
                    report(a.status, UT_ERR_HEADER, e, b);
                } else {
                    n = nn;
                }
            } else {
                report(a.status, UT_ERR_DIR, e, b);
            }
        }
        off[b] = n;
        big |= n > (uint32_t)kSmallBank;
    }
    const bool any_big = __syncthreads_or(big) != 0;
    const uint32_t total = block_exclusive_scan(off, B, sm.warp_tot);

    // Publish the aggregate at once; look back only after the event's own
    // shared-memory maps are built, so that the predecessors have had the
    // time to publish theirs.
    if (tid == 0)
        st_volatile_u64(a.tile_state + e, (e == 0 ? kFlagPrefix : kFlagAggregate) | (unsigned long long)total);
    // Events of at most map_cap hits build the shared-memory maps (sorted:
    // word positions fit 16 bits); larger bank-order events are written in
    // output order without them.
    const bool from_map = ev_ok && sm.bmap != nullptr && total <= a.map_cap && (!SORT || nw < 32768);
    const bool mapped = SORT ? from_map : ev_ok;
    if (from_map) map_event<SORT>(a, sm, evw, any_big, nw);
    if (tid < 32) {
        const unsigned long long excl = e > 0 ? lookback(a.tile_state, e, a.status, a.spin_limit) : 0ull;
        if (tid == 0) {
            if (e > 0) st_volatile_u64(a.tile_state + e, kFlagPrefix | ((excl + total) & kValueMask));
            *sm.s_base = excl;
        }
    }
    __syncthreads();
    const unsigned long long base = *sm.s_base;
    const unsigned long long end = base + total;
    const bool fits = end <= (unsigned long long)a.capacity;
    if (!fits && tid == 0) report(a.status, UT_ERR_CAPACITY, -1, -1);

    uint32_t* hit_off = a.hit_off + (size_t)e * B;
    for (int b = tid; b < B; b += nt)
        st_chk(hit_off, b, (long long)(a.n_events - e) * B + 1, (uint32_t)(base + off[b]), a.status, 108);
    if (e == a.n_events - 1 && tid == 0) a.hit_off[(size_t)a.n_events * B] = (uint32_t)end;
    if (!ev_ok) return;

    // Decode.  Mapped events are written in output order; larger ones use
    // one thread per hit (bank by binary search) writing at its ranked slot.
    if (mapped) {
        write_mapped<SORT>(a, e, sm, evw, base, total, fits, sx, sx_cap, nw, from_map);
        return;
    }
    for (uint32_t i = tid; i < total; i += nt) {
        const int b = find_bank(off, B, i);
        const uint32_t k = i - off[b];
        const uint32_t n = off[b + 1] - off[b];
        const uint16_t* w16 = bank_words(evw, b);
        const uint32_t w = ld_chk(reinterpret_cast<const uint16_t*>(evw), 2ll * ((long long)evw[b] + 1) + k,
                                  2ll * (long long)nw, a.status, 109);
        if ((w & 0x3FFu) >= (uint32_t)a.strips) report(a.status, UT_ERR_STRIP, e, b);
        uint32_t r = k;
        if (SORT) {
            if (n > (uint32_t)kSmallBank) continue;  // ranked below
            const uint32_t hk = min(half_strip(w), (uint32_t)(kKeyBins - 1));
            r = rank_small(w16, n, k, hk);
        }
        if (fits) {
            int l, s;
            bank_ls(b, S, l, s);
            write_hit(a, (uint32_t)(base + off[b] + r), l, s, w, sx, sx_cap, off[b] + r);
        }
    }
    if (SORT && fits && any_big)
        rank_big_banks(off, B, evw, sm.bigcnt, [&](int b, uint32_t pos, uint32_t, uint32_t w) {
            int l, s;
            bank_ls(b, S, l, s);
            write_hit(a, (uint32_t)(base + off[b] + pos), l, s, w, sx, sx_cap, off[b] + pos);
        });
}

}  // namespace utc

namespace utc {
// Before a block exits after a bulk copy that timed out: wait (bounded) for
// the copy still in flight so that it does not land in freed shared memory.
__device__ __forceinline__ void drain_stage(const DecodeSmem& sm, uint32_t phase, bool tma_ok, long long limit) {
    if (!tma_ok) (void)mbar_wait_bounded(sm.mbar, phase, limit);
}
}  // namespace utc
