// Greedy distance-d colouring (Algorithm 1, Section 3.1) on the device.
//
// Algorithm 1 visits the nodes in a fixed priority order (descending degree,
// ties by ascending caller node id) and gives each node the smallest colour
// not used by an earlier node within geodesic distance d.  The colour of a
// node therefore depends only on the colours of the higher-priority nodes of
// its d-ball.  The device version colours, in rounds, every node all of whose
// higher-priority d-ball neighbours are already coloured (Jones-Plassmann
// with the greedy order as priority): such a node sees exactly the colours
// the sequential sweep would have shown it, so the result is Algorithm 1's
// colouring node for node, whatever the order in which the rounds run.
//
// A node stays uncoloured while some uncoloured node of higher priority lies
// in its d-ball; such a node is remembered (the "blocker") and the ball is
// searched again only once the blocker has its colour.  The first two
// searches of a node stop at the first blocker they meet (cheap when balls
// are small); later ones walk the whole ball and keep the blocker latest in
// the greedy order, whose colouring mostly comes after the others', so that
// nodes with large balls are searched a few times rather than once per
// higher-priority neighbour.  Colours are written
// once and never change, so a node may read colours written during the same
// round: a stale "uncoloured" only postpones it to the next round, and no
// node of lower priority in its ball can be coloured before it.
//
// The d-ball is walked level by level.  For d <= 2 the levels are the CSR
// slices themselves (repeats are harmless: the test and the colour mark are
// idempotent).  For d >= 3 the nodes of levels 1..d-1 are de-duplicated in a
// per-warp open-addressing table in shared memory; a node whose ball does
// not fit is searched again in the same round by a whole CTA with a table in
// global memory (k_color_big), and one that does not fit there either sets
// the overflow flag (the caller reports the colouring as unsupported).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.h"

namespace vne {

namespace {

constexpr int kCWarps = 4;          // warps per CTA
constexpr int kWin = 1024;          // colours per mex window (32 words of 32 bits)
constexpr int kHashSlots = 2048;    // d >= 3: de-duplication table per warp
constexpr int kBallCap = 1024;      // d >= 3: nodes of levels 2..d-1 kept as frontiers

__device__ __forceinline__ int ld_color(const int32_t* p) { return __ldcg(p); }
__device__ __forceinline__ void st_color(int32_t* p, int v) { __stcg(p, v); }

__device__ __forceinline__ uint32_t hash_node(int32_t w) {
    uint32_t x = (uint32_t)w * 0x9E3779B1u;
    return x >> 21;  // 11 bits: kHashSlots = 2048
}

// The stored node of a key: its low half is the caller's id, mapped back to
// the stored numbering by inv (NULL: the numberings agree).
__device__ __forceinline__ int32_t key_node(uint64_t k, const int32_t* __restrict__ inv) {
    const int32_t id = (int32_t)(uint32_t)k;
    return inv ? __ldg(inv + id) : id;
}

// Priority key: smaller = earlier in Algorithm 1's order.
__global__ void k_color_init(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ node_id, int64_t n,
                             uint64_t* __restrict__ key, int32_t* __restrict__ inv, int32_t* __restrict__ tries,
                             int32_t* __restrict__ color, int32_t* __restrict__ blk, int32_t* __restrict__ list) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t deg = (uint32_t)(rowptr[v + 1] - rowptr[v]);
        const uint32_t id = node_id ? (uint32_t)node_id[v] : (uint32_t)v;
        key[v] = ((uint64_t)(0x7fffffffu - deg) << 32) | id;
        if (inv) inv[id] = (int32_t)v;
        tries[v] = 0;
        color[v] = -1;
        blk[v] = -1;
        list[v] = (int32_t)v;
    }
}

// Per-warp scratch in shared memory.
struct WarpScratch {
    uint32_t win[32];      // mex window bitmap
    int32_t excl[32];      // flattened enumeration: exclusive degree prefix per frontier slot
    int32_t start[32];     //   and the CSR start of each frontier node
};

struct BallCtx {
    int32_t v;
    uint64_t kv;
    int base;               // first colour of the mex window
    uint64_t bkey;          // per lane: largest key of an uncoloured higher-priority node seen, else 0
};

__device__ __forceinline__ void visit(int32_t w, const uint64_t* __restrict__ key, const int32_t* color,
                                      BallCtx& b, WarpScratch& ws) {
    const int c = ld_color(color + w);
    if (c < 0) {
        const uint64_t kw = __ldg(key + w);
        if (w != b.v && kw < b.kv && kw > b.bkey) b.bkey = kw;
    } else if (c >= b.base && c < b.base + kWin) {
        const int o = c - b.base;
        atomicOr(&ws.win[o >> 5], 1u << (o & 31));
    }
}

// Insert w into the warp's table: 1 = new, 0 = present, -1 = table full.
__device__ __forceinline__ int table_insert(int32_t* table, int32_t w) {
    uint32_t h = hash_node(w);
    for (int probe = 0; probe < kHashSlots; probe++) {
        const int32_t old = atomicCAS(&table[h], -1, w);
        if (old == -1) return 1;
        if (old == w) return 0;
        h = (h + 1) & (kHashSlots - 1);
    }
    return -1;
}

// Visit every neighbour of the `cnt` frontier nodes fr[0..cnt) with the warp
// (a flattened, load-balanced enumeration of their adjacency lists).  With a
// table, new nodes are inserted and, if `append`, stored in ball[] as the
// next frontier.  Returns true (warp-uniform) once the table overflowed or,
// with `early`, once a blocker has been seen.
__device__ __forceinline__ bool expand(const int32_t* fr, int cnt, const int32_t* __restrict__ rowptr,
                       const int32_t* __restrict__ col, const uint64_t* __restrict__ key, const int32_t* color,
                       BallCtx& b, WarpScratch& ws, int32_t* table, bool append, int32_t* ball, int* nball,
                       int* nins, bool& overflow, bool early) {
    const int lane = threadIdx.x & 31;
    for (int f0 = 0; f0 < cnt; f0 += 32) {
        const int i = f0 + lane;
        const int32_t u = i < cnt ? fr[i] : -1;
        int s = 0, deg = 0;
        if (u >= 0) {
            s = rowptr[u];
            deg = rowptr[u + 1] - s;
        }
        int inc = deg;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += t;
        }
        const int tot = __shfl_sync(0xffffffffu, inc, 31);
        ws.excl[lane] = inc - deg;
        ws.start[lane] = s;
        __syncwarp();
        for (int t0 = 0; t0 < tot; t0 += 32) {
            const int t = t0 + lane;
            if (t < tot) {
                int j = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (ws.excl[j + step] <= t) j += step;
                const int32_t w = col[ws.start[j] + t - ws.excl[j]];
                visit(w, key, color, b, ws);
                if (table) {
                    const int r = table_insert(table, w);
                    if (r < 0) {
                        overflow = true;
                    } else if (r == 1) {
                        const int q = atomicAdd(nins, 1);
                        if (q >= kHashSlots * 3 / 4) overflow = true;
                        if (append) {
                            const int pos = atomicAdd(nball, 1);
                            if (pos < kBallCap) ball[pos] = w;
                            else overflow = true;
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, overflow || (early && b.bkey != 0ull))) return true;
    }
    return false;
}

// One search of v's d-ball with mex window [base, base + kWin).  Returns the
// colour (>= 0), -1 when a blocker was found (*blocker set), -2 when the ball
// did not fit the per-warp table, -3 when every colour of the window is used.
__device__ __forceinline__ int search_ball(int32_t v, int d, int base, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const uint64_t* __restrict__ key, const int32_t* color,
                           WarpScratch& ws, int32_t* table, int32_t* ball, int* nball, int* nins, int32_t* self,
                           const int32_t* __restrict__ inv, bool early, int32_t* blocker_out) {
    const int lane = threadIdx.x & 31;
    BallCtx b{v, __ldg(key + v), base, 0ull};
    ws.win[lane] = 0u;
    const bool dedup = d >= 3;
    if (dedup) {
        for (int i = lane; i < kHashSlots; i += 32) table[i] = -1;
        if (lane == 0) {
            *nball = 0;
            *nins = 0;
            *self = v;
        }
        __syncwarp();
        if (lane == 0) table_insert(table, v);
    } else if (lane == 0) {
        *self = v;
    }
    __syncwarp();
    bool overflow = false;
    bool stop = expand(self, 1, rowptr, col, key, color, b, ws, dedup ? table : nullptr, false, ball, nball, nins,
                       overflow, early);
    if (!stop && d >= 2) {
        const int32_t rb = rowptr[v];
        stop = expand(col + rb, rowptr[v + 1] - rb, rowptr, col, key, color, b, ws, dedup ? table : nullptr, d > 2,
                      ball, nball, nins, overflow, early);
    }
    int lb = 0;
    for (int lev = 3; lev <= d && !stop; lev++) {
        __syncwarp();
        const int le = min(*nball, kBallCap);
        if (le == lb) break;  // the ball is exhausted
        // level lev - 1 lives in ball[lb, le); the new level is appended after it
        // the last level is only visited: no insertion, so the table holds
        // the nodes within distance d - 1
        stop = expand(ball + lb, le - lb, rowptr, col, key, color, b, ws, lev < d ? table : nullptr, lev < d, ball,
                      nball, nins, overflow, early);
        lb = le;
    }
    __syncwarp();
    if (__any_sync(0xffffffffu, overflow)) return -2;
    uint64_t bk = b.bkey;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const uint64_t o = __shfl_xor_sync(0xffffffffu, bk, off);
        bk = o > bk ? o : bk;
    }
    if (bk != 0ull) {
        *blocker_out = key_node(bk, inv);
        return -1;
    }
    const uint32_t word = ws.win[lane];
    const unsigned free_lanes = __ballot_sync(0xffffffffu, word != 0xffffffffu);
    if (!free_lanes) return -3;
    const int L = __ffs(free_lanes) - 1;
    const uint32_t wl = __shfl_sync(0xffffffffu, word, L);
    return base + L * 32 + (__ffs(~wl) - 1);
}

// One round over the list of uncoloured nodes.  Counters rotate over three
// slots: round r reads cnt[r % 3], appends the nodes that stay uncoloured to
// cnt[(r + 1) % 3] and clears cnt[(r + 2) % 3] (the input of round r - 1 and
// the output of round r + 1).
__global__ void __launch_bounds__(kCWarps * 32) k_color_round(ColorRound p) {
    extern __shared__ int32_t dyn[];  // d >= 3: per warp kHashSlots table + kBallCap ball
    __shared__ WarpScratch ws_all[kCWarps];
    __shared__ int nball_all[kCWarps], nins_all[kCWarps];
    __shared__ int32_t self_all[kCWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = p.round;
    int* cnt = p.cnt;
    // one thread per CTA reads the shared words (all threads reading one
    // address queue on a single L2 slice)
    __shared__ int s_total, s_over;
    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) cnt[(r + 2) % 3] = 0;
        s_total = cnt[r % 3];
        s_over = p.d >= 3 ? __ldcg(p.overflow) : 0;
    }
    __syncthreads();
    const int total = s_total;
    int* cout = cnt + (r + 1) % 3;
    if (s_over != 0) return;
    const int32_t* in = (r & 1) ? p.list[1] : p.list[0];
    int32_t* out = (r & 1) ? p.list[0] : p.list[1];
    WarpScratch& ws = ws_all[warp];
    int32_t* table = p.d >= 3 ? dyn + warp * (kHashSlots + kBallCap) : nullptr;
    int32_t* ball = p.d >= 3 ? table + kHashSlots : nullptr;
    const int nw = gridDim.x * kCWarps;
    // 32 list entries per warp step: each lane re-checks its node's blocker
    // (the common case, one load each; survivors appended with one atomic per
    // warp), then the warp searches the balls of the nodes whose blocker is
    // coloured, one after another
    const unsigned lt = (1u << lane) - 1u;
    int wmax = 0;  // colours used by this warp (max + 1), one atomicMax at the end
    for (int i0 = (blockIdx.x * kCWarps + warp) * 32; i0 < total; i0 += nw * 32) {
        // an overflow (d >= 3 only) ends the round early
        if (p.d >= 3 && __shfl_sync(0xffffffffu, lane == 0 ? __ldcg(p.overflow) : 0, 0) != 0) break;
        const int i = i0 + lane;
        int32_t v = -1;
        bool need = false;
        if (i < total) {
            v = in[i];
            const int32_t b = p.blk[v];
            need = !(b >= 0 && ld_color(p.color + b) < 0);
        }
        const unsigned stay = __ballot_sync(0xffffffffu, i < total && !need);
        if (stay) {
            int base = 0;
            if (lane == 0) base = atomicAdd(cout, __popc(stay));
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((stay >> lane) & 1u) out[base + __popc(stay & lt)] = v;
        }
        unsigned todo = __ballot_sync(0xffffffffu, need);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int32_t u = __shfl_sync(0xffffffffu, v, src);
            int base = 0, res;
            int32_t blocker = -1;
            const int tries = p.tries[u];
            for (;;) {
                res = search_ball(u, p.d, base, p.rowptr, p.col, p.key, p.color, ws, table, ball, &nball_all[warp],
                                  &nins_all[warp], &self_all[warp], p.inv, tries < 2, &blocker);
                // every colour of the window is taken: the next window (the
                // ball has at most n nodes, so this ends)
                if (res != -3 || base > (1 << 30)) break;
                base += kWin;
            }
            if (lane == 0) {
                if (res >= 0) {
                    st_color(p.color + u, res);
                    wmax = max(wmax, res + 1);
                } else if (res == -1) {
                    p.blk[u] = blocker;
                    p.tries[u] = tries + 1;
                    out[atomicAdd(cout, 1)] = u;
                } else if (p.biglist) {
                    // the ball does not fit the warp's table: the CTA-wide
                    // search of k_color_big takes the node in this round
                    p.biglist[atomicAdd(p.bigcnt + (r & 1), 1)] = u;
                } else {
                    atomicExch(p.overflow, 1);
                    out[atomicAdd(cout, 1)] = u;
                }
            }
            __syncwarp();
        }
    }
    if (lane == 0 && wmax > 0) atomicMax(p.ncolors, wmax);
}

__global__ void k_color_scatter(const int32_t* __restrict__ color, const int32_t* __restrict__ node_id, int64_t n,
                                int32_t* __restrict__ out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[node_id ? node_id[v] : v] = color[v];
}

__global__ void k_color_hist(const int32_t* __restrict__ color, int64_t n, int32_t* __restrict__ counts) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + color[v], 1);
}

// ---------------------------------------------------------------------------
// CTA-wide search for balls that do not fit a warp's table (d >= 3): the same
// level-by-level walk with 256 threads, de-duplicated in a per-CTA table in
// global memory.  Entries carry the search's epoch, so a table never needs
// clearing: an entry of an older epoch counts as empty.

constexpr int kBigThreads = 256;
constexpr int kBigTableBits = 18;
constexpr int kBigTable = 1 << kBigTableBits;  // entries per CTA
constexpr int kBigBall = 1 << 18;              // frontier nodes per CTA
constexpr int kBigWin = kBigThreads * 32;      // colours per mex window

struct BigShared {
    uint32_t win[kBigThreads];
    int32_t excl[kBigThreads];
    int32_t start[kBigThreads];
    int32_t wpre[kBigThreads / 32];
    unsigned long long bkey;
    int32_t tot, stop, overflow, nball, nins, mex, self;
    uint32_t epoch;
};

__device__ __forceinline__ int big_insert(uint64_t* tab, uint32_t epoch, int32_t w) {
    uint32_t h = ((uint32_t)w * 0x9E3779B1u) >> (32 - kBigTableBits);
    const uint64_t mine = ((uint64_t)epoch << 32) | (uint32_t)w;
    for (int probe = 0; probe < kBigTable; probe++) {
        uint64_t cur = __ldcg(reinterpret_cast<const unsigned long long*>(tab + h));
        if ((uint32_t)(cur >> 32) != epoch) {
            const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(tab + h), (unsigned long long)cur,
                                           (unsigned long long)mine);
            if (old == cur) return 1;
            cur = old;  // taken in this epoch by another thread of the CTA
        }
        if ((int32_t)(uint32_t)cur == w) return 0;
        h = (h + 1) & (kBigTable - 1);
    }
    return -1;
}

// Visit the neighbours of fr[0..cnt) with the whole CTA.  Returns true (CTA
// uniform) once the table overflowed.
__device__ __forceinline__ bool big_expand(const int32_t* fr, int cnt, const ColorRound& p, BigShared& sh, uint64_t* tab,
                           int32_t* ball, bool insert, bool append, int32_t v, uint64_t kv, int base) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t epoch = sh.epoch;
    for (int f0 = 0; f0 < cnt; f0 += kBigThreads) {
        const int i = f0 + tid;
        const int32_t u = i < cnt ? fr[i] : -1;
        int s = 0, deg = 0;
        if (u >= 0) {
            s = p.rowptr[u];
            deg = p.rowptr[u + 1] - s;
        }
        int inc = deg;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += t;
        }
        if (lane == 31) sh.wpre[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const int x0 = lane < kBigThreads / 32 ? sh.wpre[lane] : 0;
            int x = x0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += t;
            }
            if (lane < kBigThreads / 32) sh.wpre[lane] = x - x0;
            if (lane == kBigThreads / 32 - 1) sh.tot = x;
        }
        __syncthreads();
        sh.excl[tid] = inc - deg + sh.wpre[warp];
        sh.start[tid] = s;
        __syncthreads();
        const int tot = sh.tot;
        for (int t = tid; t < tot; t += kBigThreads) {
            int j = 0;
#pragma unroll
            for (int step = kBigThreads / 2; step > 0; step >>= 1)
                if (sh.excl[j + step] <= t) j += step;
            const int32_t w = p.col[sh.start[j] + t - sh.excl[j]];
            const int c = ld_color(p.color + w);
            if (c < 0) {
                const uint64_t kw = __ldg(p.key + w);
                if (w != v && kw < kv) atomicMax(&sh.bkey, (unsigned long long)kw);
            } else if (c >= base && c < base + kBigWin) {
                const int o = c - base;
                atomicOr(&sh.win[o >> 5], 1u << (o & 31));
            }
            if (insert) {
                const int r = big_insert(tab, epoch, w);
                if (r < 0) {
                    sh.overflow = 1;
                    sh.stop = 1;
                } else if (r == 1) {
                    if (atomicAdd(&sh.nins, 1) >= kBigTable / 4 * 3) {
                        sh.overflow = 1;
                        sh.stop = 1;
                    }
                    if (append) {
                        const int pos = atomicAdd(&sh.nball, 1);
                        if (pos < kBigBall) {
                            ball[pos] = w;
                        } else {
                            sh.overflow = 1;
                            sh.stop = 1;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (sh.stop) return true;
    }
    return false;
}

// Same results as search_ball: colour, -1 blocker (*blocker), -2 overflow,
// -3 window full.
__device__ __forceinline__ int big_search(int32_t v, int base, const ColorRound& p, BigShared& sh, uint64_t* tab,
                                          int32_t* ball, int32_t* blocker) {
    const int tid = threadIdx.x;
    const uint64_t kv = __ldg(p.key + v);
    if (tid == 0) {
        sh.stop = 0;
        sh.bkey = 0ull;
        sh.overflow = 0;
        sh.nball = 0;
        sh.nins = 0;
        sh.mex = 0x7fffffff;
        sh.self = v;
        sh.epoch = ++p.epoch[blockIdx.x];
        big_insert(tab, sh.epoch, v);
    }
    sh.win[tid] = 0u;
    __syncthreads();
    bool stop = big_expand(&sh.self, 1, p, sh, tab, ball, true, false, v, kv, base);
    if (!stop) {
        const int32_t rb = p.rowptr[v];
        stop = big_expand(p.col + rb, p.rowptr[v + 1] - rb, p, sh, tab, ball, p.d > 2, p.d > 2, v, kv, base);
    }
    int lb = 0;
    for (int lev = 3; lev <= p.d && !stop; lev++) {
        const int le = min(sh.nball, kBigBall);
        if (le == lb) break;
        stop = big_expand(ball + lb, le - lb, p, sh, tab, ball, lev < p.d, lev < p.d, v, kv, base);
        lb = le;
    }
    __syncthreads();
    if (sh.overflow) return -2;
    if (sh.bkey != 0ull) {
        *blocker = key_node(sh.bkey, p.inv);
        return -1;
    }
    const uint32_t word = sh.win[tid];
    if (word != 0xffffffffu) atomicMin(&sh.mex, tid * 32 + (__ffs(~word) - 1));
    __syncthreads();
    const int m = sh.mex;
    return m == 0x7fffffff ? -3 : base + m;
}

__global__ void __launch_bounds__(kBigThreads) k_color_big(ColorRound p) {
    __shared__ BigShared sh;
    const int r = p.round;
    int* bc = p.bigcnt;
    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) bc[(r + 1) & 1] = 0;
        sh.tot = bc[r & 1];
        sh.stop = __ldcg(p.overflow);
    }
    __syncthreads();
    const int total = sh.tot;
    if (total == 0 || sh.stop != 0) return;
    __syncthreads();  // sh.tot and sh.stop are reused by the searches
    int* cout = p.cnt + (r + 1) % 3;
    int32_t* out = (r & 1) ? p.list[0] : p.list[1];
    uint64_t* tab = p.bigtab + (size_t)blockIdx.x * kBigTable;
    int32_t* ball = p.bigball + (size_t)blockIdx.x * kBigBall;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        if (threadIdx.x == 0) sh.stop = __ldcg(p.overflow);
        __syncthreads();
        if (sh.stop) break;
        __syncthreads();
        const int32_t v = p.biglist[i];
        int base = 0, res;
        int32_t blocker = -1;
        for (;;) {
            res = big_search(v, base, p, sh, tab, ball, &blocker);
            if (res != -3 || base > (1 << 30)) break;
            base += kBigWin;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (res >= 0) {
                st_color(p.color + v, res);
                atomicMax(p.ncolors, res + 1);
            } else {
                if (res == -1) p.blk[v] = blocker;
                else atomicExch(p.overflow, 1);
                out[atomicAdd(cout, 1)] = v;
            }
        }
        __syncthreads();
    }
}

int sm_count() {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    return sms;
}

int flat_grid(int64_t n) {
    const int64_t want = (n + 255) / 256, cap = (int64_t)sm_count() * 8;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace

cudaError_t launch_color_init(const int32_t* rowptr, const int32_t* node_id, int64_t n, uint64_t* key,
                              int32_t* inv, int32_t* tries, int32_t* color, int32_t* blk, int32_t* list,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_color_init<<<flat_grid(n), 256, 0, st>>>(rowptr, node_id, n, key, inv, tries, color, blk, list);
    return cudaGetLastError();
}

size_t color_round_smem(int d) { return d >= 3 ? (size_t)kCWarps * (kHashSlots + kBallCap) * sizeof(int32_t) : 0; }

cudaError_t launch_color_round(const ColorRound& p, cudaStream_t st) {
    const size_t smem = color_round_smem(p.d);
    if (smem) {
        cudaError_t e = cudaFuncSetAttribute(k_color_round, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = sm_count() * (p.d >= 3 ? 4 : 8);
    k_color_round<<<grid, kCWarps * 32, smem, st>>>(p);
    return cudaGetLastError();
}

int color_big_ctas() { return sm_count(); }
size_t color_big_table_entries() { return (size_t)kBigTable; }
size_t color_big_ball_entries() { return (size_t)kBigBall; }

cudaError_t launch_color_big(const ColorRound& p, cudaStream_t st) {
    k_color_big<<<color_big_ctas(), kBigThreads, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_color_scatter(const int32_t* color, const int32_t* node_id, int64_t n, int32_t* out,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_color_scatter<<<flat_grid(n), 256, 0, st>>>(color, node_id, n, out);
    return cudaGetLastError();
}

cudaError_t launch_color_hist(const int32_t* color, int64_t n, int32_t* counts, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_color_hist<<<flat_grid(n), 256, 0, st>>>(color, n, counts);
    return cudaGetLastError();
}

}  // namespace vne
