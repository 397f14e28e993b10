// dvc_pool.cuh -- the fused search step: several trees per CTA in lockstep.
//
// A CTA owns T trees (its slots) and W warps.  Every kDetAhead iterations all
// threads sample the next kDetAhead determinizations of every slot, one
// thread each (a determinization depends only on the root view, the seed, the
// tree and the iteration).  One iteration of every tree the CTA owns runs as:
//   1. tree phase -- warp w walks slots w, w+W, ...: take the iteration's
//      determinization, descend by UCB1, expand one child, and publish the leaf;
//   2. playout phase -- the P playouts of every published leaf form one pool;
//      each lane takes the next playout of the pool as soon as its previous one
//      ends (one guess, plus the draw that follows, per loop step), so lanes stay
//      busy until the pool is empty;
//   3. backprop -- each warp adds its trees' playout results along their paths.
// Trees stay strictly sequential (iteration i+1 sees i's statistics), which is
// what makes results bit-exact with the single-threaded oracle, while every
// lane of the CTA does useful work in every phase.  Trees with spent budgets
// drop out of phase 1 and keep helping with phase 2, so uneven budgets balance
// inside a CTA; across CTAs the host assigns trees by total work.
#pragma once
#include "dvc_tree.cuh"

namespace dvc {

constexpr int kPathMax = 20;
constexpr int kDetAhead = 64;  // determinizations sampled ahead per tree

struct ForestDev {
    const dvc_state* roots;
    TreeMeta* meta;
    const DetPlan* plans;
    const unsigned long long* tables;
    Node* nodes;
    int32_t* link;
    int32_t* created;
    float2* ucb;  // per slot: wins/n, 1/sqrt(n)
    float* csl;   // per slot: c * sqrt(ln n)
    int32_t* flags;
    unsigned long long* words;
    uint4* set_key;    // vanilla: plausible-set tables of all trees (TreeMeta::set_off)
    int32_t* set_slot;
};

__device__ __forceinline__ SetTable set_table(const ForestDev& F, const TreeMeta& tm) {
    return SetTable{F.set_key + tm.set_off, F.set_slot + tm.set_off, (uint32_t)tm.set_cells};
}

__device__ __forceinline__ void latch_error(int32_t* flags, int32_t code) { atomicCAS(&flags[0], 0, code); }

// Shared-memory layout of one CTA with T slots and W warps.
struct PoolLayout {
    uint32_t pl, meta, root, leaf, path, mover, wins, misc, base, E, cnt, bytes;
    __host__ __device__ PoolLayout(int T, int W) {
        uint32_t o = 0;
        auto take = [&](uint32_t n) {
            const uint32_t at = o;
            o += (n + 15u) & ~15u;
            return at;
        };
        pl = take(sizeof(DetPlan) * T);
        meta = take(sizeof(TreeMeta) * T);
        root = take(32u * T);
        leaf = take(32u * T);
        path = take(4u * kPathMax * T);
        mover = take((uint32_t)kPathMax * T);
        wins = take(16u * T);
        misc = take(16u * T);  // per slot: np, end, tree index, 0
        base = take(4u * T);   // per slot: first iteration sampled ahead
        E = take(4u * 104u * W);
        cnt = take(4u * 8u);   // [parity][nleaf, next, ntrees, 0]
        bytes = o;
    }
};

// ORD: the ordering-aware playout policy (sp.policy == 1), compiled apart so
// that the uniform playout loop keeps its registers.
// det_ahead / tree0_ahead: kDetAhead determinized roots and first in-tree
// stream blocks per tree (the forest's pipeline buffers; rewritten at the
// start of every launch).
template <int MAXT, bool FAST2, bool ORD = false>
__global__ void __launch_bounds__(MAXT, 1)
    mcts_pool_kernel(ForestDev F, SearchParams sp, int n_iter, const int32_t* order, int n_trees, int T,
                     dvc_state* det_ahead, uint4* tree0_ahead) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_magic[32];
    __shared__ unsigned long long s_lut12[FAST2 ? 4096 : 1];
    const int W = (int)(blockDim.x >> 5);
    const PoolLayout L(T, W);
    DetPlan* s_pl = (DetPlan*)(smem + L.pl);
    TreeMeta* s_tm = (TreeMeta*)(smem + L.meta);
    dvc_state* s_root = (dvc_state*)(smem + L.root);
    dvc_state* s_leaf = (dvc_state*)(smem + L.leaf);
    int32_t* s_path = (int32_t*)(smem + L.path);
    uint8_t* s_mover = (uint8_t*)(smem + L.mover);
    int32_t* s_wins = (int32_t*)(smem + L.wins);
    int32_t* s_misc = (int32_t*)(smem + L.misc);
    int32_t* s_base = (int32_t*)(smem + L.base);
    uint32_t* s_E = (uint32_t*)(smem + L.E);
    int32_t* s_cnt = (int32_t*)(smem + L.cnt);

    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const int base = blockIdx.x * T;
    const int nslot = min(T, n_trees - base);
    if (nslot <= 0) return;

    // load the slots
    for (int s = (int)warp; s < nslot; s += W) {
        const int t = order ? order[base + s] : base + s;
        if (lane == 0) {
            s_tm[s] = F.meta[t];
            s_pl[s] = F.plans[t];
            s_root[s] = F.roots[t];
            TreeMeta& tm = s_tm[s];
            const bool usable = s_pl[s].ok && s_pl[s].total && !tm.failed;
            s_misc[4 * s + 0] = 0;
            s_misc[4 * s + 1] = usable ? min(tm.budget, tm.done + n_iter) : tm.done;
            s_misc[4 * s + 2] = t;
        }
    }
    if (tid < 8) s_cnt[tid] = 0;
    fill_magic(s_magic, tid, blockDim.x);
    if constexpr (FAST2) fill_select12(s_lut12, tid, blockDim.x);
    __syncthreads();

    uint32_t words = 0u, nsteps = 0u;  // per lane; summed in 64 bits per warp at the end
    for (int iter = 0;; ++iter) {
        int32_t* cnt = s_cnt + 4 * (iter & 1);
        if (iter % kDetAhead == 0) {
            // ---- 0. the next kDetAhead determinizations of every running slot
            __syncthreads();
            for (int idx = (int)tid; idx < nslot * kDetAhead; idx += (int)blockDim.x) {
                const int s = idx / kDetAhead, k = idx - s * kDetAhead;
                const TreeMeta& tm = s_tm[s];
                if (k == 0) s_base[s] = tm.done;
                if (tm.done + k >= s_misc[4 * s + 1]) continue;
                const uint32_t it = (uint32_t)(tm.done + k);
                const size_t a = (size_t)s_misc[4 * s + 2] * kDetAhead + (size_t)k;
                const G root = load_state(s_root[s]);
                Rng dr;
                dr.open(sp.seed, tm.tree_id, 0u, it, kTagDet);
                G det;
                det_sample(s_pl[s], F.tables + tm.table_off, root, dr, det);
                dvc_state ds;
                store_state(det, ds);
                det_ahead[a] = ds;
                Rng tr;
                tr.open(sp.seed, tm.tree_id, 0u, it, kTagTree);
                tree0_ahead[a] = tr.block0();
            }
            __syncthreads();
        }
        // ---- 1. tree phase
        for (int s = (int)warp; s < nslot; s += W) {
            TreeMeta& tm = s_tm[s];
            if (tm.done >= s_misc[4 * s + 1]) continue;
            const uint32_t it = (uint32_t)tm.done;
            Node* nodes = F.nodes + tm.node_off;
            int32_t* link = F.link + tm.node_off;
            int32_t* created = F.created + tm.node_off;
            const G root = load_state(s_root[s]);
            const size_t a = (size_t)s_misc[4 * s + 2] * kDetAhead + (it - (uint32_t)s_base[s]);
            const G det = load_state(det_ahead[a]);
            Descent d;
            int32_t* path = s_path + s * kPathMax;
            uint8_t* mover = s_mover + s * kPathMax;
            const SetTable st = set_table(F, tm);
            descend(det, root.cur, nodes, link, F.ucb + tm.node_off, F.csl + tm.node_off, tm, sp, it, path, mover,
                    s_E + warp * 104u, d, tree0_ahead + a, st);
            bool ok = true;
            if (d.found) {
                int32_t next_free = tm.next_free, used = tm.used;
                ok = expand_child(d, nodes, link, created, tm, next_free, used, it, path, mover, sp.tree_continue != 0,
                                  st);
                if (lane == 0) {
                    tm.next_free = next_free;
                    tm.used = used;
                }
            }
            if (lane == 0) {
                if (!ok) {
                    tm.failed = 1;
                    s_misc[4 * s + 1] = tm.done;  // stop this tree
                    latch_error(F.flags, DVC_E_OOM);
                } else {
                    s_misc[4 * s + 0] = d.np;
                    store_state(d.s, s_leaf[s]);
                    int32_t* w = s_wins + 4 * s;
                    w[0] = w[1] = w[2] = w[3] = 0;
                    if (d.s.winner < 4u) w[d.s.winner] = sp.playouts;  // finished in the tree
                    atomicAdd(&cnt[2], 1);
                }
            }
        }
        __syncthreads();
        if (cnt[2] == 0) break;
        if (tid == 0) {
            int32_t* other = s_cnt + 4 * ((iter + 1) & 1);
            other[0] = other[1] = other[2] = 0;
            // list of leaves that need playouts: slots with a fresh, unfinished leaf
            int32_t n = 0;
            for (int s = 0; s < nslot; ++s)
                if (s_tm[s].done < s_misc[4 * s + 1] && s_leaf[s].winner == kNone) s_misc[4 * (n++) + 3] = s;
            cnt[0] = n;
        }
        __syncthreads();
        // ---- 2. playout phase: P playouts of each listed leaf, handed to lanes as they free up
        {
            const int P = sp.playouts;
            const int total = cnt[0] * P;
            int slot = 0, steps = 0;
            WordQueue r;
            // state of the lane's current game
            G g;    // general path, ordering-aware policy
            GR gr;  // general path, uniform policy
            uint32_t h0 = 0, h1 = 0, rev = 0, cur = 0, drawn = kNone, winner = kNone;
            auto start = [&](int p) {
                const int k = p / P;
                slot = s_misc[4 * k + 3];
                const dvc_state& ls = s_leaf[slot];
                r.open(sp.seed, s_tm[slot].tree_id, (uint32_t)(p - k * P), (uint32_t)s_tm[slot].done, kTagRoll);
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
                // a may-stop leaf's first continue coin is a game step of its
                // own (the fast path counts it as an iteration of its loop)
                steps = (!FAST2 && (ls.flags & 2u)) ? 1 : 0;
            };
            int p = atomicAdd(&cnt[1], 1);
            bool busy = p < total;
            if (busy) start(p);
            while (__any_sync(0xFFFFFFFFu, busy)) {
                if (busy) {
                    int res;
                    if constexpr (FAST2) {
                        if (winner == kPend)
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
                    if (res == kGameOver || steps >= 128) {
                        // at most |T| guesses per game: 128 steps is a broken invariant
                        if (res != kGameOver) latch_error(F.flags, DVC_E_INTERNAL);
                        const uint32_t w = res == kGameOver ? winner : kNone;
                        if (w < 4u) atomicAdd(&s_wins[4 * slot + (int)w], 1);
                        words += r.used();
                        nsteps += steps;
                        p = atomicAdd(&cnt[1], 1);
                        busy = p < total;
                        if (busy) start(p);
                    }
                }
            }
        }
        __syncthreads();
        // ---- 3. backprop
        for (int s = (int)warp; s < nslot; s += W) {
            TreeMeta& tm = s_tm[s];
            if (tm.done >= s_misc[4 * s + 1]) continue;
            backprop(F.nodes + tm.node_off, F.ucb + tm.node_off, F.csl + tm.node_off, s_path + s * kPathMax,
                     s_mover + s * kPathMax, s_misc[4 * s + 0], s_wins + 4 * s, sp.playouts, sp.c_uct);
            __syncwarp();
            if (lane == 0) tm.done += 1;
            __syncwarp();
        }
    }
    // write the slots back
    for (int s = (int)warp; s < nslot; s += W) {
        if (lane == 0) {
            TreeMeta& dst = F.meta[s_misc[4 * s + 2]];
            dst.done = s_tm[s].done;
            dst.next_free = s_tm[s].next_free;
            dst.used = s_tm[s].used;
            dst.failed = s_tm[s].failed;
        }
    }
    if (F.words) {  // F.words[0]: random words, F.words[1]: game steps (guesses)
        const unsigned long long sum = warp_sum_u64((unsigned long long)words);
        const unsigned long long st = warp_sum_u64((unsigned long long)nsteps);
        if (lane == 0 && sum) atomicAdd(F.words, sum);
        if (lane == 0 && st) atomicAdd(F.words + 1, st);
    }
}

}  // namespace dvc
