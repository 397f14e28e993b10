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

// Finish the previous iteration of tree t (backprop) and run its next
// selection and expansion.
// Trees order[i0 .. i1-1], one warp each.
__global__ void __launch_bounds__(128)
    pipe_select_kernel(ForestDev F, SearchParams sp, int i0, int i1, const int32_t* order, PipeBufs P) {
    __shared__ uint32_t s_E[4][104];
    const int i = i0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= i1) return;
    const int t = order[i];
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
    Rng dr;
    dr.open(sp.seed, tm.tree_id, 0u, it, kTagDet);
    G det;
    det_sample(F.plans[t], F.tables + tm.table_off, root, dr, det);
    Descent d;
    int32_t* path = P.path + (size_t)t * kPathMax;
    uint8_t* mover = P.mover + (size_t)t * kPathMax;
    descend(det, root.cur, nodes, link, F.ucb + tm.node_off, F.csl + tm.node_off, tm, sp, it, path, mover, s_E[wl],
            d);
    bool ok = true;
    int32_t next_free = tm.next_free, used = tm.used;
    if (d.found) ok = expand_child(d, nodes, link, F.created + tm.node_off, tm, next_free, used, it, path, mover);
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
template <bool FAST2>
__global__ void __launch_bounds__(1024, 1)
    pipe_rollout_kernel(SearchParams sp, int n, int L, int b0, const int32_t* order, const TreeMeta* meta, PipeBufs P,
                        unsigned long long* words_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_magic[32];
    __shared__ unsigned long long s_lut12[FAST2 ? 4096 : 1];
    __shared__ int32_t s_n, s_next;
    int32_t* s_tree = (int32_t*)smem;       // listed leaves: tree index
    int32_t* s_wins = s_tree + L;           // 4 per listed leaf
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
    const int Pp = sp.playouts;
    const int total = nl * Pp;
    unsigned long long words = 0ull;
    int k = 0, steps = 0;
    WordQueue r;
    G g;
    uint32_t h0 = 0, h1 = 0, rev = 0, cur = 0, drawn = kNone, winner = kNone;
    auto start = [&](int p) {
        k = p / Pp;
        const dvc_state& ls = s_leaf[k];
        if constexpr (FAST2) {
            h0 = ls.hand[0];
            h1 = ls.hand[1];
            rev = ls.revealed;
            cur = ls.cur;
            drawn = ls.drawn;
            winner = kNone;
        } else {
            g = load_state(ls);
        }
        r.open(sp.seed, s_tid[k], (uint32_t)(p - k * Pp), s_it[k], kTagRoll);
        steps = 0;
    };
    int p = atomicAdd(&s_next, 1);
    bool busy = p < total;
    if (busy) start(p);
    while (__any_sync(0xFFFFFFFFu, busy)) {
        if (busy) {
            int res;
            if constexpr (FAST2) {
                res = step_2p24(h0, h1, rev, cur, drawn, winner, r, sp.cont_thr, s_magic, s_lut12);
            } else {
                r.ensure(4);
                res = random_guess(g, r, sp.cont_thr, s_magic);
                if (res == kTurnOver) next_turn(g, r);
                winner = g.winner;
            }
            ++steps;
            if (res == kGameOver || steps >= 128) {
                const uint32_t w = res == kGameOver ? winner : kNone;
                if (w < 4u) atomicAdd(&s_wins[4 * k + (int)w], 1);
                words += r.used();
                p = atomicAdd(&s_next, 1);
                busy = p < total;
                if (busy) start(p);
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
    }
    if (words_out) {
        const unsigned long long sum = warp_sum_u64(words);
        if (lane == 0 && sum) atomicAdd(words_out, sum);
    }
}

// The last iteration's backprop of a step.
__global__ void __launch_bounds__(128) pipe_backprop_kernel(ForestDev F, SearchParams sp, int n, PipeBufs P) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= n) return;
    pipe_apply_pending(F, sp, t, P);
}

// Value mode: the network's win probabilities stand in for the playouts of
// every fresh, unfinished leaf -- each seat is credited round(p * P) of the P
// visits (a leaf that ended inside the tree keeps its exact credit).
__global__ void pipe_value_wins_kernel(int n, PipeBufs P, const float* probs, int playouts) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (P.np[t] < 0 || P.leaf[t].winner != kNone) return;
    int32_t* w = P.wins + 4 * t;
    for (int s = 0; s < 4; ++s) w[s] = (int32_t)(probs[4 * t + s] * (float)playouts + 0.5f);
}

__host__ __device__ inline uint32_t pipe_rollout_smem(int L) {
    return (uint32_t)(4 * L + 16 * L + 4 * L + 4 * L + 16 + 32 * L);
}

}  // namespace dvc
