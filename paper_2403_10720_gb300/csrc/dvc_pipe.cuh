// dvc_pipe.cuh -- the search iteration as launches over the whole forest,
// chained in a CUDA graph:
//   pipe_select   one warp per tree: backpropagate the previous iteration's
//                 playout results, then determinize, descend, expand and
//                 publish the next leaf;
//   pipe_rollout  one CTA per group of trees: the P playouts of the group's leaves
//                 form one pool that lanes draw from as they free up;
//   pipe_backprop after the last iteration of a step: the pending backprop.
// The tree walk needs many registers and the playout loop few, so giving each
// its own kernel lets the playouts run at full occupancy.  Every tree still
// runs its iterations strictly in order, so results equal the fused kernel's
// and the oracle's bit for bit.
#pragma once
#include "dvc_pool.cuh"

namespace dvc {

struct PipeBufs {
    dvc_state* leaf;    // per tree
    int32_t* path;      // per tree, kPathMax slots
    uint8_t* mover;     // per tree, kPathMax seats
    int32_t* np;        // per tree: path length, -1 if the tree does not run this iteration
    int32_t* wins;      // per tree, 4 seats
    int32_t* step_end;  // per tree: iteration at which this step stops
    dvc_state* det;     // per tree, kDetAhead determinized roots: iterations det_base .. det_base + kDetAhead - 1
    uint4* tree0;       // per tree, kDetAhead first blocks of the iterations' tree streams (tag 3)
    int32_t* det_base;  // per tree; far below zero (bytes 0xC0) when nothing is sampled ahead
    int32_t* flags;     // the context's latched error
};

__global__ void pipe_begin_kernel(ForestDev F, int n, int n_iter, int32_t* step_end) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const TreeMeta tm = F.meta[t];
    const DetPlan& pl = F.plans[t];
    const bool usable = pl.ok && pl.total && !tm.failed;
    step_end[t] = usable ? min(tm.budget, tm.done + n_iter) : tm.done;
}

// Backpropagate the path the previous iteration left (np >= 0), if any.
__device__ __forceinline__ void pipe_apply_pending(ForestDev& F, const SearchParams& sp, int t, PipeBufs& P) {
    const int32_t np = P.np[t];
    if (np < 0) return;
    TreeMeta& tm = F.meta[t];
    const long long off = tm.node_off;
    backprop(F.nodes + off, F.ucb + off, F.csl + off, P.path + (size_t)t * kPathMax, P.mover + (size_t)t * kPathMax,
             np, P.wins + 4 * t, sp.playouts, sp.c_uct);
    __syncwarp();
    if ((threadIdx.x & 31u) == 0) {
        tm.done += 1;
        P.np[t] = -1;
    }
    __syncwarp();
}

// A determinization depends only on the root view, the seed, the tree id and
// the iteration (stream tag 2), not on the tree's statistics, so the next
// `count` of them are sampled up front, one thread per (tree, iteration),
// instead of on the tree walk's critical path.  Trees order[i0 .. i1-1]
// (trees i0 .. i1-1 if order is null).
__global__ void __launch_bounds__(128)
    pipe_det_kernel(ForestDev F, SearchParams sp, int i0, int i1, const int32_t* order, PipeBufs P, int count) {
    const int g = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int i = i0 + g / count, k = g % count;
    if (i >= i1) return;
    const int t = order ? order[i] : i;
    const TreeMeta& tm = F.meta[t];
    // the tree's next select first applies its pending backprop (done + 1)
    const int32_t base = tm.done + (P.np[t] >= 0 ? 1 : 0);
    if (k == 0) P.det_base[t] = base;
    if (base + k >= P.step_end[t]) return;
    const G root = load_state(F.roots[t]);
    Rng dr;
    dr.open(sp.seed, tm.tree_id, 0u, (uint32_t)(base + k), kTagDet);
    G det;
    det_sample(F.plans[t], F.tables + tm.table_off, root, dr, det);
    dvc_state s;
    store_state(det, s);
    P.det[(size_t)t * kDetAhead + k] = s;
    Rng tr;  // the iteration's in-tree draws start from this block
    tr.open(sp.seed, tm.tree_id, 0u, (uint32_t)(base + k), kTagTree);
    P.tree0[(size_t)t * kDetAhead + k] = tr.block0();
}

// Finish the previous iteration of tree t (backprop) and run its next
// selection and expansion.
// Trees order[i0 .. i1-1] (trees i0 .. i1-1 if order is null), one warp each.
// VANILLA: the trees have a plausible-set layer (compiled apart, so that the
// MCTS-dvc walk carries none of its code).
template <bool VANILLA>
__global__ void __launch_bounds__(128)
    pipe_select_kernel(ForestDev F, SearchParams sp, int i0, int i1, const int32_t* order, PipeBufs P) {
    __shared__ uint32_t s_E[4][104];
    const int i = i0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= i1) return;
    const int t = order ? order[i] : i;
    const uint32_t lane = threadIdx.x & 31u, wl = (threadIdx.x >> 5) & 3u;
    pipe_apply_pending(F, sp, t, P);
    TreeMeta& tmr = F.meta[t];
    const TreeMeta tm = tmr;
    if (tm.done >= P.step_end[t]) {
        if (lane == 0) P.np[t] = -1;
        return;
    }
    const uint32_t it = (uint32_t)tm.done;
    Node* nodes = F.nodes + tm.node_off;
    int32_t* link = F.link + tm.node_off;
    const G root = load_state(F.roots[t]);
    G det;
    const uint32_t ahead = it - (uint32_t)P.det_base[t];
    const uint4* tree0 = nullptr;
    if (ahead < (uint32_t)kDetAhead) {
        det = load_state(P.det[(size_t)t * kDetAhead + ahead]);
        tree0 = P.tree0 + (size_t)t * kDetAhead + ahead;
    } else {
        Rng dr;
        dr.open(sp.seed, tm.tree_id, 0u, it, kTagDet);
        det_sample(F.plans[t], F.tables + tm.table_off, root, dr, det);
    }
    Descent d;
    int32_t* path = P.path + (size_t)t * kPathMax;
    uint8_t* mover = P.mover + (size_t)t * kPathMax;
    const SetTable st = VANILLA ? set_table(F, tm) : SetTable{nullptr, nullptr, 0u};
    descend(det, root.cur, nodes, link, F.ucb + tm.node_off, F.csl + tm.node_off, tm, sp, it, path, mover, s_E[wl],
            d, tree0, st);
    bool ok = true;
    int32_t next_free = tm.next_free, used = tm.used;
    if (d.found)
        ok = expand_child(d, nodes, link, F.created + tm.node_off, tm, next_free, used, it, path, mover,
                          sp.tree_continue != 0, st);
    if (lane == 0) {
        tmr.next_free = next_free;
        tmr.used = used;
        int32_t* w = P.wins + 4 * t;
        w[0] = w[1] = w[2] = w[3] = 0;
        if (!ok) {
            tmr.failed = 1;
            P.step_end[t] = tm.done;
            P.np[t] = -1;
            latch_error(F.flags, DVC_E_OOM);
        } else {
            P.np[t] = d.np;
            dvc_state s;
            store_state(d.s, s);
            P.leaf[t] = s;
            if (d.s.winner < 4u) w[d.s.winner] = sp.playouts;  // finished inside the tree
        }
    }
}

// Trees order[b*L .. b*L+L-1] belong to CTA b; this launch runs CTAs b0 + blockIdx.x.
// The CTA's L x P playouts form one pool: a lane whose game ends takes the
// next playout index (warp-aggregated: one shared-memory atomic per warp and
// step), so lanes wait for the longest game only at the end of the pool.
// Every lane queues its words in a shared-memory ring (RingQueue), refilled
// warp-wide, so that the Philox rounds run for most lanes at once; for
// two-player 24-tile games it also lets two 1024-thread CTAs fit on an SM.
// ORD: the ordering-aware playout policy (sp.policy == 1), compiled apart.
// PEND: leaves may begin where the mover may stop (the full game tree, or
// d_max = 0); without it that check is compiled out of the playout loop,
// since an in-tree action always clears the may-stop bit otherwise.
// CNT: keep the work counters (random words, game steps) in words_out;
// compiled out for forests that switched counting off.
// Registers: 32 for the two-player path (two 1024-thread or three
// 512-thread CTAs per SM, with room left in the register file for the
// other chains' tree walks), up to 64 for the general path.
template <bool FAST2, bool ORD = false, bool PEND = true, bool CNT = true>
__global__ void __launch_bounds__(1024, FAST2 ? 2 : 1)
    pipe_rollout_kernel(SearchParams sp, int n, int L, int b0, const int32_t* order, const TreeMeta* meta, PipeBufs P,
                        unsigned long long* words_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_magic[32];
    __shared__ unsigned long long s_lut12[FAST2 ? 4096 : 1];
    __shared__ int32_t s_n, s_next;
    uint32_t* s_ring = (uint32_t*)smem;                   // 16 words per thread
    int32_t* s_tree = (int32_t*)(smem + 64u * blockDim.x);  // listed leaves: tree index
    int32_t* s_wins = s_tree + L;                                  // 4 per listed leaf
    uint32_t* s_tid = (uint32_t*)(s_wins + 4 * L);
    uint32_t* s_it = s_tid + L;
    dvc_state* s_leaf = (dvc_state*)(((uintptr_t)(s_it + L) + 15) & ~(uintptr_t)15);
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    fill_magic(s_magic, tid, blockDim.x);
    if constexpr (FAST2) fill_select12(s_lut12, tid, blockDim.x);
    if (tid == 0) {
        int32_t k = 0;
        for (int e = 0; e < L; ++e) {
            const int i = (b0 + (int)blockIdx.x) * L + e;
            if (i >= n) break;
            const int t = order[i];
            if (P.np[t] < 0 || P.leaf[t].winner != kNone) continue;
            s_tree[k] = t;
            k++;
        }
        s_n = k;
        s_next = 0;
    }
    __syncthreads();
    const int nl = s_n;
    for (int k = (int)tid; k < nl; k += (int)blockDim.x) {
        const int t = s_tree[k];
        s_leaf[k] = P.leaf[t];
        s_tid[k] = meta[t].tree_id;
        s_it[k] = (uint32_t)meta[t].done;
        s_wins[4 * k] = s_wins[4 * k + 1] = s_wins[4 * k + 2] = s_wins[4 * k + 3] = 0;
    }
    __syncthreads();
    const uint32_t Pp = (uint32_t)sp.playouts;
    const uint32_t total = (uint32_t)nl * Pp;
    // playout p belongs to leaf p / Pp: multiply-high by ceil(2^32 / Pp) gives
    // the quotient or one more (p < 2^32), fixed by one comparison
    const uint32_t mP = Pp > 1u ? 0xFFFFFFFFu / Pp + 1u : 0u;
    // work counters: random words per lane; game steps per warp (every
    // running lane takes one step per pass of the loop)
    uint32_t words = 0u, wsteps = 0u;
    uint32_t k = 0, steps = 0;
    RingQueue r;
    r.ring = s_ring + tid;
    r.stride = blockDim.x;
    G g;    // general path, ordering-aware policy
    GR gr;  // general path, uniform policy
    uint32_t h0 = 0, h1 = 0, rev = 0, cur = 0, drawn = kNone, winner = kNone;
    auto start = [&](uint32_t p) {
        k = Pp > 1u ? __umulhi(p, mP) : p;
        if (k * Pp > p) --k;
        const dvc_state& ls = s_leaf[k];
        r.open(sp.seed, s_tid[k], p - k * Pp, s_it[k], kTagRoll);
        if constexpr (FAST2) {
            h0 = ls.hand[0];
            h1 = ls.hand[1];
            rev = ls.revealed;
            cur = ls.cur;
            drawn = ls.drawn;
            winner = (ls.flags & 2u) ? kPend : kNone;  // may stop: continue coin first
        } else {
            g = load_state(ls);
            playout_begin(g, r, sp.cont_thr);
            if constexpr (!ORD) gr = to_gr(g);
        }
        // a may-stop leaf's first continue coin is a game step of its own
        // (the fast path counts it as an iteration of its loop)
        steps = (!FAST2 && (ls.flags & 2u)) ? 1u : 0u;
    };
    // the lanes in `want` take consecutive playout indices (all lanes call);
    // once a take comes back short the pool is empty for good (dry, warp-uniform)
    bool dry = false;
    auto take = [&](bool want) -> uint32_t {
        const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
        uint32_t base = 0;
        if (m) {
            const int leader = __ffs(m) - 1;
            if ((int)lane == leader) base = (uint32_t)atomicAdd(&s_next, __popc(m));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            dry = base + (uint32_t)__popc(m) >= total;
        }
        return base + (uint32_t)__popc(m & ((1u << lane) - 1u));
    };
    uint32_t p = take(true);
    bool busy = p < total;
    if (busy) start(p);
    for (;;) {
        const unsigned running = __ballot_sync(0xFFFFFFFFu, busy);
        if (!running) break;
        if constexpr (CNT) wsteps += __popc(running);
        bool ended = false;
        if (busy) {
            int res;
            if constexpr (FAST2) {
                if (PEND && winner == kPend)
                    res = step_2p24_pending(h0, h1, cur, drawn, winner, r, sp.cont_thr, s_lut12);
                else if constexpr (ORD)
                    res = step_2p24_ordered(h0, h1, rev, cur, drawn, winner, r, sp.cont_thr, s_lut12);
                else
                    res = step_2p24(h0, h1, rev, cur, drawn, winner, r, sp.cont_thr, s_magic, s_lut12);
            } else if constexpr (ORD) {
                r.ensure(4);
                res = random_guess_ordered(g, r, sp.cont_thr);
                if (res == kTurnOver) next_turn(g, r);
                winner = g.winner;
            } else {
                res = step_gen(gr, r, sp.cont_thr, s_magic);
                winner = gr.winner;
            }
            ++steps;
            if (res == kGameOver || steps >= 128u) {
                // a game has at most |T| guesses (each turns one tile face up), so
                // 128 steps means a broken invariant: nobody is credited, and the
                // leaf's wins fall short of P (checked below)
                const uint32_t w = res == kGameOver ? winner : kNone;
                if (w < 4u) atomicAdd(&s_wins[4 * k + w], 1);
                if constexpr (CNT) words += r.used();
                ended = true;
            }
        }
        if (dry) {
            busy = busy && !ended;
        } else if (__any_sync(0xFFFFFFFFu, ended)) {
            const uint32_t q = take(ended);
            if (ended) {
                busy = q < total;
                if (busy) start(q);
            }
        }
    }
    __syncthreads();
    for (int e = (int)tid; e < nl; e += (int)blockDim.x) {
        int32_t* w = P.wins + 4 * s_tree[e];
        w[0] = s_wins[4 * e];
        w[1] = s_wins[4 * e + 1];
        w[2] = s_wins[4 * e + 2];
        w[3] = s_wins[4 * e + 3];
        if (s_wins[4 * e] + s_wins[4 * e + 1] + s_wins[4 * e + 2] + s_wins[4 * e + 3] != (int32_t)Pp)
            latch_error(P.flags, DVC_E_INTERNAL);
    }
    if (CNT && words_out) {  // words_out[0]: random words, words_out[1]: game steps (guesses)
        const unsigned long long sum = warp_sum_u64((unsigned long long)words);
        if (lane == 0 && sum) atomicAdd(words_out, sum);
        if (lane == 0 && wsteps) atomicAdd(words_out + 1, (unsigned long long)wsteps);
        if constexpr (PEND && !FAST2) {
            // the general path draws a may-stop leaf's first continue coin when
            // a playout starts, outside the loop counted above: one step each
            if (tid == 0) {
                unsigned long long coins = 0ull;
                for (int e = 0; e < nl; ++e) coins += (s_leaf[e].flags & 2u) ? Pp : 0u;
                if (coins) atomicAdd(words_out + 1, coins);
            }
        }
    }
}

// Dynamic shared memory of pipe_rollout_kernel: the word rings and the
// listed leaves.
__host__ __device__ inline uint32_t pipe_rollout_smem(int L, int threads) {
    return (uint32_t)(64 * threads + 4 * L + 16 * L + 4 * L + 4 * L + 16 + 32 * L);
}

// Lane compaction for the two-player 24-tile playouts (uniform policy, no
// may-stop leaves), a variant of pipe_rollout_kernel measured against it
// and off by default.  Warps 0 .. R-1 receive, the others donate: once the
// CTA's pool of playouts is empty, a donor warp with at most `donate_at`
// games still running posts them (state, leaf, stream position) to a mailbox
// in shared memory and leaves the playout loop; receiver lanes that are idle
// take posted games and finish them.  Every game goes on with the same words
// of its own stream, so results equal the default kernel's.  Receivers stop
// once no donor is left and the mailbox is drained; every wait is bounded
// (DVC_E_TIMEOUT latched if a limit is hit).
constexpr int kMailFields = 11;

__host__ __device__ inline uint32_t pipe_compact_smem(int L, int threads, int receivers) {
    const uint32_t cap = (uint32_t)(threads / 32 - receivers) * 32u;
    return pipe_rollout_smem(L, threads) + cap * 4u * (kMailFields + 1u);
}

__global__ void __launch_bounds__(1024, 2)
    pipe_rollout_compact_kernel(SearchParams sp, int n, int L, int b0, const int32_t* order, const TreeMeta* meta,
                                PipeBufs P, unsigned long long* words_out, int R, int donate_at) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_magic[32];
    __shared__ unsigned long long s_lut12[4096];
    __shared__ int32_t s_n, s_next, s_posted, s_taken, s_donors;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    uint32_t* s_ring = (uint32_t*)smem;
    int32_t* s_tree = (int32_t*)(smem + 64u * blockDim.x);
    int32_t* s_wins = s_tree + L;
    uint32_t* s_tid = (uint32_t*)(s_wins + 4 * L);
    uint32_t* s_it = s_tid + L;
    dvc_state* s_leaf = (dvc_state*)(((uintptr_t)(s_it + L) + 15) & ~(uintptr_t)15);
    const uint32_t cap = (blockDim.x >> 5) * 32u - (uint32_t)R * 32u;
    uint32_t* mail = (uint32_t*)(smem + pipe_rollout_smem(L, blockDim.x));  // kMailFields x cap, then cap flags
    volatile uint32_t* ready = mail + kMailFields * cap;
    fill_magic(s_magic, tid, blockDim.x);
    fill_select12(s_lut12, tid, blockDim.x);
    for (uint32_t e = tid; e < cap; e += blockDim.x) ready[e] = 0u;
    if (tid == 0) {
        int32_t k = 0;
        for (int e = 0; e < L; ++e) {
            const int i = (b0 + (int)blockIdx.x) * L + e;
            if (i >= n) break;
            const int t = order[i];
            if (P.np[t] < 0 || P.leaf[t].winner != kNone) continue;
            s_tree[k] = t;
            k++;
        }
        s_n = k;
        s_next = 0;
        s_posted = 0;
        s_taken = 0;
        s_donors = (int)(blockDim.x >> 5) - R;
    }
    __syncthreads();
    const int nl = s_n;
    for (int k = (int)tid; k < nl; k += (int)blockDim.x) {
        const int t = s_tree[k];
        s_leaf[k] = P.leaf[t];
        s_tid[k] = meta[t].tree_id;
        s_it[k] = (uint32_t)meta[t].done;
        s_wins[4 * k] = s_wins[4 * k + 1] = s_wins[4 * k + 2] = s_wins[4 * k + 3] = 0;
    }
    __syncthreads();
    const uint32_t Pp = (uint32_t)sp.playouts;
    const uint32_t total = (uint32_t)nl * Pp;
    const uint32_t mP = Pp > 1u ? 0xFFFFFFFFu / Pp + 1u : 0u;
    const bool receiver = (int)warp < R;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t words = 0u, wsteps = 0u;  // random words per lane, game steps per warp
    uint32_t k = 0, steps = 0;
    RingQueue r;
    r.ring = s_ring + tid;
    r.stride = blockDim.x;
    uint32_t h0 = 0, h1 = 0, rev = 0, cur = 0, drawn = kNone, winner = kNone;
    auto start = [&](uint32_t p) {
        k = Pp > 1u ? __umulhi(p, mP) : p;
        if (k * Pp > p) --k;
        const dvc_state& ls = s_leaf[k];
        r.open(sp.seed, s_tid[k], p - k * Pp, s_it[k], kTagRoll);
        h0 = ls.hand[0];
        h1 = ls.hand[1];
        rev = ls.revealed;
        cur = ls.cur;
        drawn = ls.drawn;
        winner = kNone;
        steps = 0;
    };
    auto take = [&](bool want) -> uint32_t {
        const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
        uint32_t base = 0;
        if (m) {
            const int leader = __ffs(m) - 1;
            if ((int)lane == leader) base = (uint32_t)atomicAdd(&s_next, __popc(m));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
        }
        return base + (uint32_t)__popc(m & lt);
    };
    uint32_t p = take(true);
    bool busy = p < total;
    if (busy) start(p);
    bool timed_out = false;
    for (uint32_t guard = 0;; ++guard) {
        if (guard > (1u << 24)) {  // far beyond any CTA's playouts: give up, report
            timed_out = true;
            break;
        }
        wsteps += __popc(__ballot_sync(0xFFFFFFFFu, busy));
        bool ended = false;
        if (busy) {
            const int res = step_2p24(h0, h1, rev, cur, drawn, winner, r, sp.cont_thr, s_magic, s_lut12);
            ++steps;
            if (res == kGameOver || steps >= 128u) {  // 128 steps: a broken invariant, checked below
                const uint32_t w = res == kGameOver ? winner : kNone;
                if (w < 4u) atomicAdd(&s_wins[4 * k + w], 1);
                words += r.used();
                ended = true;
            }
        }
        if (__any_sync(0xFFFFFFFFu, ended)) {
            const uint32_t q = take(ended);
            if (ended) {
                busy = q < total;
                if (busy) start(q);
            }
        }
        // shared counters are read by lane 0 and broadcast: every branch
        // below is taken by the whole warp
        int32_t next = 0, posted = 0, taken = 0, donors = 0;
        if (lane == 0) {
            // donors first: once it reads 0 every post is made, so the posted
            // count read after it is final
            donors = *(volatile int32_t*)&s_donors;
            __threadfence_block();
            next = *(volatile int32_t*)&s_next;
            posted = *(volatile int32_t*)&s_posted;
            taken = *(volatile int32_t*)&s_taken;
        }
        next = __shfl_sync(0xFFFFFFFFu, next, 0);
        posted = __shfl_sync(0xFFFFFFFFu, posted, 0);
        taken = __shfl_sync(0xFFFFFFFFu, taken, 0);
        donors = __shfl_sync(0xFFFFFFFFu, donors, 0);
        const bool pool_empty = next >= (int32_t)total;
        const unsigned running = __ballot_sync(0xFFFFFFFFu, busy);
        if (!receiver) {
            if (!pool_empty) continue;
            if (running == 0u) break;
            if (__popc(running) > donate_at) continue;
            // donate the running games and leave
            const int leader = __ffs(running) - 1;
            uint32_t base = 0;
            if ((int)lane == leader) base = (uint32_t)atomicAdd(&s_posted, __popc(running));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (busy) {
                const uint32_t e = base + (uint32_t)__popc(running & lt);
                const uint32_t v[kMailFields] = {h0, h1, rev, cur, drawn, k, steps, r.k1, r.j, r.i, r.head};
#pragma unroll
                for (int f = 0; f < kMailFields; ++f) mail[f * cap + e] = v[f];
                __threadfence_block();
                ready[e] = 1u;
            }
            busy = false;
            break;
        }
        // receiver: idle lanes take posted games
        if (!pool_empty) continue;
        const unsigned idle = ~running;
        if (posted > taken && idle) {
            const int leader = __ffs(idle) - 1;
            int32_t base = 0, cnt = 0;
            if ((int)lane == leader) {
                cnt = min(__popc(idle), posted - taken);
                if (atomicCAS(&s_taken, taken, taken + cnt) != taken) cnt = 0;  // another warp took first
                base = taken;
            }
            cnt = __shfl_sync(0xFFFFFFFFu, cnt, leader);
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            const int rank = __popc(idle & lt);
            if (!busy && rank < cnt) {
                const uint32_t e = (uint32_t)(base + rank);
                uint32_t spin = 0;
                while (ready[e] == 0u && spin < (1u << 22)) ++spin;  // the donor sets it right after writing
                if (ready[e] == 0u) {
                    timed_out = true;
                } else {
                    __threadfence_block();
                    h0 = mail[0 * cap + e];
                    h1 = mail[1 * cap + e];
                    rev = mail[2 * cap + e];
                    cur = mail[3 * cap + e];
                    drawn = mail[4 * cap + e];
                    k = mail[5 * cap + e];
                    steps = mail[6 * cap + e];
                    r.k0 = (uint32_t)sp.seed;
                    r.tw = kTagRoll + 16u * (uint32_t)(sp.seed >> 32);
                    r.k1 = mail[7 * cap + e];
                    r.j = mail[8 * cap + e];
                    r.i = mail[9 * cap + e];
                    r.resume(mail[10 * cap + e]);
                    winner = kNone;
                    busy = true;
                }
            }
            if (__any_sync(0xFFFFFFFFu, timed_out)) break;
            continue;
        }
        if (running != 0u) continue;
        // nothing running here: done once no donor can still post and every post is taken
        if (donors == 0 && posted == taken) break;
        __nanosleep(64);
    }
    if (timed_out && lane == 0) latch_error(P.flags, DVC_E_TIMEOUT);
    if (!receiver) {
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            atomicSub(&s_donors, 1);
        }
    }
    __syncthreads();
    for (int e = (int)tid; e < nl; e += (int)blockDim.x) {
        int32_t* w = P.wins + 4 * s_tree[e];
        w[0] = s_wins[4 * e];
        w[1] = s_wins[4 * e + 1];
        w[2] = s_wins[4 * e + 2];
        w[3] = s_wins[4 * e + 3];
        if (s_wins[4 * e] + s_wins[4 * e + 1] + s_wins[4 * e + 2] + s_wins[4 * e + 3] != (int32_t)Pp)
            latch_error(P.flags, DVC_E_INTERNAL);
    }
    if (words_out) {  // words_out[0]: random words, words_out[1]: game steps (guesses)
        const unsigned long long sum = warp_sum_u64((unsigned long long)words);
        if (lane == 0 && sum) atomicAdd(words_out, sum);
        if (lane == 0 && wsteps) atomicAdd(words_out + 1, (unsigned long long)wsteps);
    }
}

// The last iteration's backprop of a step.
__global__ void __launch_bounds__(128) pipe_backprop_kernel(ForestDev F, SearchParams sp, int n, PipeBufs P) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= n) return;
    pipe_apply_pending(F, sp, t, P);
}

// Value mode: the network's win probabilities stand in for the playouts of
// every fresh, unfinished leaf of trees t0 .. t1-1 -- each seat is credited
// round(p * P) of the P visits (a leaf that ended inside the tree keeps its
// exact credit).
__global__ void pipe_value_wins_kernel(int t0, int t1, PipeBufs P, const float* probs, int playouts) {
    const int t = t0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (t >= t1) return;
    if (P.np[t] < 0 || P.leaf[t].winner != kNone) return;
    int32_t* w = P.wins + 4 * t;
    for (int s = 0; s < 4; ++s) w[s] = (int32_t)(probs[4 * t + s] * (float)playouts + 0.5f);
}

}  // namespace dvc
