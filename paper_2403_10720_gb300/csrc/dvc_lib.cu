// dvc_lib.cu -- kernels and the C ABI of libdvc (see include/dvc.h).
#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <deque>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "dvc_internal.h"
#include "dvc_pipe.cuh"

using namespace dvc;
using namespace dvc_host;

namespace {
constexpr int kMaxChains = 32;  // independent chains of the pipeline graph
constexpr int kValueChains = 16;  // at most, in value mode (each chain pads its leaves to 128 rows)

// Default launch shape of an engine for n trees on `sms` SMs with P playouts
// per leaf.  Pipeline: small rollout CTAs of at least two trees, warps enough
// for one playout per thread (4 to 16), and as many chains (up to 16) as give
// each chain about 0.85 CTAs per SM, so that the tree walks of some chains
// run beside the playouts of the others.  Fused: every SM holds a CTA, one
// warp per tree up to 16.
void default_shape(int n, int sms, int engine, int P, int& T, int& W, int& chains) {
    const int S = std::max(sms, 1);
    if (engine == 2) {
        chains = std::max(1, std::min(24, (int)std::lround(n / (1.12 * S))));
        T = std::max(2, std::min(64, (int)std::ceil(n / (chains * 0.85 * S))));
        W = std::max(4, std::min(16, (T * std::max(P, 1) + 31) / 32));
    } else {
        // a warp per tree, and enough warps for one playout per thread (16 at most)
        T = std::max(1, std::min(32, (n + S - 1) / S));
        W = std::min(16, std::max(T, (T * std::max(P, 1) + 31) / 32));
        chains = 1;
    }
}
}  // namespace

struct dvc_forest {
    dvc_ctx* ctx;
    int n;
    uint64_t seed;
    std::vector<int32_t> h_budgets;
    dvc_state* roots;
    TreeMeta* meta;
    DetPlan* plans;
    unsigned long long* tables;
    Node* nodes;
    int32_t* link;
    int32_t* created;
    long long total_slots;
    uint32_t table_cap;
    // split-step state
    Descent* work;
    int32_t* paths;   // n x 20
    uint8_t* movers;  // n x 20
    dvc_state* leaves;
    uint32_t* leaf_tree;
    uint32_t* leaf_iter;
    unsigned long long* d_words;
    int32_t* export_scratch;
    int32_t export_cap;
    int32_t* order;          // tree order: CTAs get equal total budget
    int trees_per_cta;       // trees per CTA (fused kernel and pipeline rollouts)
    int warps_per_cta;       // 0: default
    int engine;              // 1: fused lockstep kernel, 2: three-kernel pipeline
    float2* ucb;
    float* csl;
    uint4* set_key;      // vanilla: plausible-set tables (2 * budget cells per tree)
    int32_t* set_slot;
    PipeBufs pipe;
    cudaStream_t cap_stream;  // capture stream for the pipeline graph
    cudaStream_t chain_stream[kMaxChains - 1];  // chains 2.. of the pipeline graph (chain 1 runs on cap_stream)
    cudaEvent_t fork_ev, join_ev[kMaxChains - 1];
    cudaGraphExec_t chunk_exec;  // pipeline graph of kChunkIters iterations (captured on first use)
    cudaGraphExec_t value_exec;  // the same for value mode
    dvc_value_rows vrows;        // value mode: network activations, one slice per chain
    int chains;               // independent chains in the pipeline graph (1..32)
    float* probs;             // value mode: win probabilities per tree
    int active_prefix;        // fused engine: only trees [0, active_prefix) of the order run (servers)
    int cmp_receivers;        // lane compaction in the pipeline's two-player playouts: receiver warps (0 = off)
    int cmp_donate_at;        // ... and the running games at or below which a donor warp hands its games over
    int no_count;             // work counters off (dvc_forest_count_work)
};

namespace {

constexpr int kDetChunk = 256;

__device__ __forceinline__ void latch(int32_t* flags, int32_t code) { atomicCAS(&flags[0], 0, code); }

// ------------------------------------------------------------------ kernels

__global__ void philox_kernel(int n, const uint32_t* ctr, const uint32_t* key, uint32_t* out, int ref) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t a = ctr[4 * i], b = ctr[4 * i + 1], c = ctr[4 * i + 2], d = ctr[4 * i + 3];
    if (ref) {
        uint4 cc = make_uint4(a, b, c, d);
        uint2 kk = make_uint2(key[2 * i], key[2 * i + 1]);
        uint4 r = curand_Philox4x32_10(cc, kk);
        a = r.x; b = r.y; c = r.z; d = r.w;
    } else {
        philox10(a, b, c, d, key[2 * i], key[2 * i + 1]);
    }
    out[4 * i] = a;
    out[4 * i + 1] = b;
    out[4 * i + 2] = c;
    out[4 * i + 3] = d;
}

// Root generation: deal, random history of d draws, then the mover draws.
__global__ void init_kernel(dvc_config cfg, uint64_t seed, int n, dvc_state* out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    Rng r;
    r.open(seed, (uint32_t)idx, 0u, 0u, kTagInit);
    const uint32_t np = (uint32_t)cfg.nplayers;
    const uint32_t tmask = cfg.ntiles >= 26 ? 0x03FFFFFFu : 0x00FFFFFFu;
    for (int attempt = 0; attempt < 16; ++attempt) {
        G g;
        g.h0 = g.h1 = g.h2 = g.h3 = 0u;
        g.rev = 0u;
        g.jg0 = g.jg1 = g.jflag = g.mstop = 0u;
        g.drawn = kNone;
        g.alive = (1u << np) - 1u;
        g.winner = kNone;
        g.np = np;
        g.tmask = tmask;
        for (uint32_t p = 0; p < np; ++p) {
            g.cur = p;
            for (int d = 0; d < cfg.deal; ++d) draw(g, r);
        }
        g.drawn = kNone;
        g.cur = 0;
        uint32_t target = pick(r.next(), (uint32_t)cfg.max_predraw + 1u);
        const bool last = attempt == 15;
        if (last) target = 0;
        uint32_t draws = 0;
        bool over = false;
        while (draws < target && g.pool()) {
            draw(g, r);
            ++draws;
            for (;;) {
                const int res = random_guess(g, r, cfg.cont_thr);
                if (res == kGameOver) {
                    over = true;
                    break;
                }
                if (res == kTurnOver) break;
            }
            if (over) break;
            g.cur = next_alive(g.alive, g.cur, np);
        }
        if (over) continue;
        bool bad = false;
        for (uint32_t p = 0; p < np; ++p) bad |= __popc(g.hand(p) & g.rev) > cfg.max_revealed;
        if (bad && !last) continue;
        draw(g, r);
        store_state(g, out[idx]);
        return;
    }
}

// One thread per root: plan, fill its table in a private workspace slot, sample.
__global__ void determinize_kernel(const dvc_state* roots, int n, int observer, uint64_t seed,
                                   const uint32_t* tree_ids, const uint32_t* iter_ids, dvc_state* out,
                                   unsigned long long* ws, int32_t* flags) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const G g = load_state(roots[idx]);
    const uint32_t obs = observer < 0 ? g.cur : (uint32_t)observer;
    DetPlan pl;
    det_plan(g, obs, pl);
    if (!pl.ok) {
        latch(flags, DVC_E_UNSUPPORTED);
        out[idx] = roots[idx];
        return;
    }
    unsigned long long* F = ws + (size_t)(idx % kDetChunk) * kDetMaxCells;
    det_fill(pl, F, 0u, 1u, [] {});
    Rng r;
    r.open(seed, tree_ids[idx], 0u, iter_ids[idx], kTagDet);
    G o;
    det_sample(pl, F, g, r, o);
    store_state(o, out[idx]);
}

// One self-play move per game: the guess actions[i] on the true state, then
// the next seat's draw on stream (seed, game id, turn, tag 5).
__global__ void play_move_kernel(dvc_state* states, int n, const int32_t* actions, uint64_t seed,
                                 const uint32_t* game_ids, uint32_t turn, bool cont, int32_t* flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t code = actions[i];
    G g = load_state(states[i]);
    if (code < 0 || g.winner != kNone) return;  // no move, or the game is over
    const uint32_t c = (uint32_t)code;
    if (c > kStop || !action_legal(g, c)) {
        atomicCAS(&flags[0], 0, DVC_E_INVALID);
        return;
    }
    Rng tr;
    tr.open(seed, game_ids ? game_ids[i] : (uint32_t)i, 0u, turn, kTagPlay);
    tree_apply(g, c, tr, cont);
    store_state(g, states[i]);
}

// Leaf-parallel playouts: thread -> (leaf, playout).  Win counts are summed
// with integer atomics, so the result is independent of scheduling.
template <bool ORD>
__global__ void rollout_kernel(const dvc_state* leaves, int n_leaves, int P, uint64_t seed,
                               const uint32_t* tree_ids, const uint32_t* leaf_ids, uint32_t cont_thr, int32_t* wins,
                               unsigned long long* words, int32_t* flags) {
    __shared__ uint32_t s_magic[32];
    fill_magic(s_magic, threadIdx.x, blockDim.x);
    __syncthreads();
    const long long total = (long long)n_leaves * P;
    unsigned long long my_words = 0ull;
    for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(gid / P);
        const int j = (int)(gid - (long long)l * P);
        const dvc_state ls = leaves[l];
        uint32_t winner;
        if (ls.winner != kNone) {
            winner = ls.winner;
        } else {
            G g = load_state(ls);
            WordQueue r;
            r.open(seed, tree_ids[l], (uint32_t)j, leaf_ids[l], kTagRoll);
            playout_begin(g, r, cont_thr);
            winner = kNone;
            if constexpr (ORD) {
                for (int guard = 0; guard < 128; ++guard) {
                    r.ensure(4);
                    const int res = random_guess_ordered(g, r, cont_thr);
                    if (res == kGameOver) {
                        winner = g.winner;
                        break;
                    }
                    if (res == kTurnOver) next_turn(g, r);
                }
            } else {
                GR gr = to_gr(g);
                for (int guard = 0; guard < 128; ++guard) {
                    if (step_gen(gr, r, cont_thr, s_magic) == kGameOver) {
                        winner = gr.winner;
                        break;
                    }
                }
            }
            // at most |T| guesses per game: no winner after 128 is a broken invariant
            if (winner == kNone) latch_error(flags, DVC_E_INTERNAL);
            my_words += r.used();
        }
        if (winner < 4u) atomicAdd(&wins[4 * l + (int)winner], 1);
    }
    if (words) {
        const unsigned long long s = warp_sum_u64(my_words);
        if ((threadIdx.x & 31u) == 0 && s) atomicAdd(words, s);
    }
}



// Split steps: one warp per tree for select and expand, results kept in
// global memory between launches.
__global__ void mcts_select_kernel(ForestDev F, SearchParams sp, int n, Descent* work, int32_t* paths,
                                   uint8_t* movers) {
    __shared__ uint32_t s_E[4][104];
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t wl = (threadIdx.x >> 5) & 3u;
    if (t >= n) return;
    const TreeMeta tm = F.meta[t];
    Descent& d = work[t];
    const uint32_t lane = threadIdx.x & 31u;
    if (tm.done >= tm.budget || tm.failed || !F.plans[t].ok || !F.plans[t].total) {
        if (lane == 0) d.np = -1;
        return;
    }
    const G root = load_state(F.roots[t]);
    Rng dr;
    dr.open(sp.seed, tm.tree_id, 0u, (uint32_t)tm.done, kTagDet);
    G det;
    det_sample(F.plans[t], F.tables + tm.table_off, root, dr, det);
    Descent dd;
    descend(det, root.cur, F.nodes + tm.node_off, F.link + tm.node_off, F.ucb + tm.node_off, F.csl + tm.node_off, tm,
            sp, (uint32_t)tm.done, paths + (size_t)t * kPathMax, movers + (size_t)t * kPathMax, s_E[wl], dd, nullptr,
            set_table(F, tm));
    if (lane == 0) d = dd;
}

__global__ void mcts_expand_kernel(ForestDev F, int n, Descent* work, int32_t* paths, uint8_t* movers,
                                   dvc_state* leaves, uint32_t* leaf_tree, uint32_t* leaf_iter, bool cont) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= n) return;
    const uint32_t lane = threadIdx.x & 31u;
    TreeMeta& tmr = F.meta[t];
    const TreeMeta tm = tmr;
    Descent d = work[t];
    if (d.np < 0) {
        if (lane == 0) {
            dvc_state s = {};
            s.winner = 0xFE;
            leaves[t] = s;
            leaf_tree[t] = tm.tree_id;
            leaf_iter[t] = (uint32_t)tm.done;
        }
        return;
    }
    int32_t next_free = tm.next_free;
    int32_t used = tm.used;
    bool ok = true;
    if (d.found)
        ok = expand_child(d, F.nodes + tm.node_off, F.link + tm.node_off, F.created + tm.node_off, tm, next_free,
                          used, (uint32_t)tm.done, paths + (size_t)t * kPathMax, movers + (size_t)t * kPathMax, cont,
                          set_table(F, tm));
    if (lane == 0) {
        tmr.next_free = next_free;
        tmr.used = used;
        if (!ok) {
            tmr.failed = 1;
            latch(F.flags, DVC_E_OOM);
            d.np = -1;
        }
        work[t] = d;
        dvc_state s;
        store_state(d.s, s);
        if (!ok) s.winner = 0xFE;
        leaves[t] = s;
        leaf_tree[t] = tm.tree_id;
        leaf_iter[t] = (uint32_t)tm.done;
    }
}

__global__ void mcts_backprop_kernel(ForestDev F, SearchParams sp, int n, const Descent* work, const int32_t* paths,
                                     const uint8_t* movers, const int32_t* wins) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= n) return;
    const Descent& d = work[t];
    if (d.np < 0) return;
    TreeMeta& tm = F.meta[t];
    backprop(F.nodes + tm.node_off, F.ucb + tm.node_off, F.csl + tm.node_off, paths + (size_t)t * kPathMax,
             movers + (size_t)t * kPathMax, d.np, wins + 4 * t, sp.playouts, sp.c_uct);
    __syncwarp();
    if ((threadIdx.x & 31u) == 0) tm.done += 1;
}

__global__ void root_stats_kernel(ForestDev F, int n, int32_t* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const TreeMeta tm = F.meta[t];
    const Node* nodes = F.nodes + tm.node_off;
    const G root = load_state(F.roots[t]);
    const Node r = nodes[0];
    const uint32_t nchild = r.meta >> 12;
    int32_t best = -1, bv = 0, bw = 0;
    uint32_t brank = 0xFFFFFFFFu;
    int32_t blk = r.child;
    uint32_t seen = 0, k = 0;
    while (seen < nchild) {
        const uint32_t size = block_size(k, true, (uint32_t)tm.root_legal);
        const uint32_t cnt = min(size, nchild - seen);
        for (uint32_t e = 0; e < cnt; ++e) {
            const Node c = nodes[blk + (int32_t)e];
            const uint32_t code = c.meta & 0xFFFu;
            const uint32_t rk = canon_rank(code, root.cur, root.np);
            if (best < 0 || c.visits > bv || (c.visits == bv && rk < brank)) {
                best = (int32_t)code;
                bv = c.visits;
                bw = c.wins;
                brank = rk;
            }
        }
        seen += cnt;
        ++k;
        if (seen < nchild) blk = F.link[tm.node_off + blk];
    }
    int32_t* o = out + 8 * t;
    o[0] = best;
    o[1] = bv;
    o[2] = bw;
    o[3] = r.visits;
    o[4] = (int32_t)nchild;
    o[5] = tm.used;
    o[6] = tm.done;
    o[7] = tm.failed;
}

// Vanilla MCTS-dvc decision (one CTA per tree): an action's visits and wins
// summed over every plausible set's child with that action; most visits
// wins, ties to the lowest canonical rank.  Root children = sets.
__global__ void __launch_bounds__(256) root_stats_vanilla_kernel(ForestDev F, int n, int32_t* out) {
    __shared__ int32_t s_v[4096], s_w[4096];
    __shared__ unsigned long long s_best;
    const int t = blockIdx.x;
    if (t >= n) return;
    const uint32_t tid = threadIdx.x;
    for (uint32_t a = tid; a < 4096u; a += blockDim.x) s_v[a] = s_w[a] = 0;
    if (tid == 0) s_best = 0ull;
    __syncthreads();
    const TreeMeta tm = F.meta[t];
    const Node* nodes = F.nodes + tm.node_off;
    const int32_t* link = F.link + tm.node_off;
    const G root = load_state(F.roots[t]);
    const Node r = nodes[0];
    const uint32_t nsets = r.meta >> 12;
    for (uint32_t i = tid; i < nsets; i += blockDim.x) {
        const Node sn = nodes[r.child + (int32_t)i];
        const uint32_t nchild = sn.meta >> 12;
        int32_t blk = sn.child;
        uint32_t seen = 0, k = 0;
        while (seen < nchild) {
            const uint32_t size = block_size(k, false, 0u);
            const uint32_t cnt = min(size, nchild - seen);
            for (uint32_t e = 0; e < cnt; ++e) {
                const Node c = nodes[blk + (int32_t)e];
                const uint32_t code = c.meta & 0xFFFu;
                atomicAdd(&s_v[code], c.visits);
                atomicAdd(&s_w[code], c.wins);
            }
            seen += cnt;
            ++k;
            if (seen < nchild) blk = link[blk];
        }
    }
    __syncthreads();
    // order key: visits, then the complement of the canonical rank (< 2^13), then the code
    unsigned long long best = 0ull;
    for (uint32_t a = tid; a < 4096u; a += blockDim.x) {
        if (s_v[a] <= 0) continue;
        const unsigned long long key = (unsigned long long)(uint32_t)s_v[a] << 32 |
                                       (unsigned long long)(0x1FFFu - canon_rank(a, root.cur, root.np)) << 12 | a;
        best = key > best ? key : best;
    }
    if (best) atomicMax(&s_best, best);
    __syncthreads();
    if (tid == 0) {
        const unsigned long long b = s_best;
        const int32_t code = b ? (int32_t)(b & 0xFFFu) : -1;
        int32_t* o = out + 8 * t;
        o[0] = code;
        o[1] = b ? s_v[code] : 0;
        o[2] = b ? s_w[code] : 0;
        o[3] = r.visits;
        o[4] = (int32_t)nsets;
        o[5] = tm.used;
        o[6] = tm.done;
        o[7] = tm.failed;
    }
}

// Export of one tree in creation order (row 0 = root).  Nodes carry the
// iteration that created them; at most one node is created per iteration, so
// a node's row is 1 + the number of iterations before its own that created a
// node.  iter_rank holds one int per iteration of the tree's budget.
// Root-parallel merge (Sec. III-B): group g is trees g*K .. g*K+K-1, all
// searched from one root with their own streams; each action's root visits
// and wins are summed over the group's trees (for vanilla trees over every
// plausible set of each tree too) and the decision is the action with most
// visits, ties to the lowest canonical rank.  One CTA per group.
__global__ void __launch_bounds__(256) root_merge_kernel(ForestDev F, int K, int groups, int vanilla, int32_t* out) {
    __shared__ int32_t s_v[4096], s_w[4096];
    __shared__ unsigned long long s_best;
    __shared__ int32_t s_tot[4];  // root visits, iterations done, failed, distinct actions
    const int g = blockIdx.x;
    if (g >= groups) return;
    const uint32_t tid = threadIdx.x;
    for (uint32_t a = tid; a < 4096u; a += blockDim.x) s_v[a] = s_w[a] = 0;
    if (tid < 4) s_tot[tid] = 0;
    if (tid == 0) s_best = 0ull;
    __syncthreads();
    const dvc_state r0 = F.roots[g * K];
    for (int k = 0; k < K; ++k) {
        const int t = g * K + k;
        const TreeMeta tm = F.meta[t];
        const Node* nodes = F.nodes + tm.node_off;
        const int32_t* link = F.link + tm.node_off;
        const Node r = nodes[0];
        if (tid == 0) {
            const dvc_state rt = F.roots[t];
            bool same = true;
            for (int i = 0; i < 8; ++i)
                same &= reinterpret_cast<const uint32_t*>(&rt)[i] == reinterpret_cast<const uint32_t*>(&r0)[i];
            if (!same) latch(F.flags, DVC_E_INVALID);  // a group must share its root
            s_tot[0] += r.visits;
            s_tot[1] += tm.done;
            s_tot[2] |= tm.failed;
        }
        // the nodes whose children are summed: the root, or every set node of a vanilla root
        const uint32_t nparents = vanilla ? (r.meta >> 12) : 1u;
        for (uint32_t pi = 0; pi < nparents; ++pi) {
            const Node pn = vanilla ? nodes[r.child + (int32_t)pi] : r;
            const uint32_t nchild = pn.meta >> 12;
            int32_t blk = pn.child;
            uint32_t seen = 0, kb = 0;
            while (seen < nchild) {
                const uint32_t size = block_size(kb, !vanilla, (uint32_t)tm.root_legal);
                const uint32_t cnt = min(size, nchild - seen);
                for (uint32_t e = tid; e < cnt; e += blockDim.x) {
                    const Node c = nodes[blk + (int32_t)e];
                    const uint32_t code = c.meta & 0xFFFu;
                    atomicAdd(&s_v[code], c.visits);
                    atomicAdd(&s_w[code], c.wins);
                }
                seen += cnt;
                ++kb;
                if (seen < nchild) blk = link[blk];
            }
        }
    }
    __syncthreads();
    const G root = load_state(r0);
    unsigned long long best = 0ull;
    int32_t distinct = 0;
    for (uint32_t a = tid; a < 4096u; a += blockDim.x) {
        if (s_v[a] <= 0) continue;
        ++distinct;
        const unsigned long long key = (unsigned long long)(uint32_t)s_v[a] << 32 |
                                       (unsigned long long)(0x1FFFu - canon_rank(a, root.cur, root.np)) << 12 | a;
        best = key > best ? key : best;
    }
    if (best) atomicMax(&s_best, best);
    if (distinct) atomicAdd(&s_tot[3], distinct);
    __syncthreads();
    if (tid == 0) {
        const unsigned long long b = s_best;
        const int32_t code = b ? (int32_t)(b & 0xFFFu) : -1;
        int32_t* o = out + 8 * g;
        o[0] = code;
        o[1] = b ? s_v[code] : 0;
        o[2] = b ? s_w[code] : 0;
        o[3] = s_tot[0];
        o[4] = s_tot[3];
        o[5] = K;
        o[6] = s_tot[1];
        o[7] = s_tot[2];
    }
}

__global__ void export_flag_kernel(ForestDev F, int t, int32_t* iter_rank) {
    const TreeMeta tm = F.meta[t];
    const int32_t* created = F.created + tm.node_off;
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < tm.next_free; s += gridDim.x * blockDim.x)
        if (s > 0 && created[s] >= 0) iter_rank[created[s]] = 1;
}

__global__ void export_scan_kernel(int32_t n, int32_t* iter_rank) {
    int32_t acc = 1;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t f = iter_rank[i];
        iter_rank[i] = f ? acc : -1;
        acc += f;
    }
}

__global__ void export_rows_kernel(ForestDev F, int t, const int32_t* iter_rank, int32_t rows, int32_t* out) {
    const TreeMeta tm = F.meta[t];
    const Node* nodes = F.nodes + tm.node_off;
    const int32_t* link = F.link + tm.node_off;
    const int32_t* created = F.created + tm.node_off;
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < tm.next_free; p += gridDim.x * blockDim.x) {
        if (p != 0 && created[p] < 0) continue;
        const int32_t prow = p == 0 ? 0 : iter_rank[created[p]];
        const Node nd = nodes[p];
        if (prow < rows) {
            out[4 * prow + 0] = p == 0 ? 0 : (int32_t)(nd.meta & 0xFFFu);
            if (p == 0) out[1] = -1;
            out[4 * prow + 2] = nd.visits;
            out[4 * prow + 3] = nd.wins;
        }
        const uint32_t nchild = nd.meta >> 12;
        int32_t blk = nd.child;
        uint32_t seen = 0, k = 0;
        while (seen < nchild) {
            const uint32_t size = block_size(k, p == 0, (uint32_t)tm.root_legal);
            const uint32_t cnt = min(size, nchild - seen);
            for (uint32_t e = 0; e < cnt; ++e) {
                const int32_t crow = iter_rank[created[blk + (int32_t)e]];
                if (crow < rows) out[4 * crow + 1] = prow;
            }
            seen += cnt;
            ++k;
            if (seen < nchild) blk = link[blk];
        }
    }
}

// (Re)initialise tree t (one warp): plan the root view's determinization, fill
// its counting table, count the root's legal guesses, reset it to a lone root.
__device__ void init_tree(ForestDev& F, int t, DetPlan* plans, unsigned long long* tables, uint32_t table_cap,
                          int nplayers, int ntiles, int32_t* pipe_np) {
    const uint32_t lane = threadIdx.x & 31u;
    dvc_state* roots = const_cast<dvc_state*>(F.roots);
    const G g = load_state(roots[t]);
    DetPlan& pl = plans[t];
    if (lane == 0) {
        det_plan(g, g.cur, pl);
        pl.ok = pl.cells <= table_cap ? 1u : 0u;
    }
    __syncwarp();
    TreeMeta& tm = F.meta[t];
    if (pl.ok) det_fill(pl, tables + tm.table_off, lane, 32u, [] { __syncwarp(); });
    if (lane == 0) {
        const dvc_state& rs = roots[t];
        const bool variant = rs.nplayers == nplayers && rs.ntiles == ntiles;  // the context's game
        const bool usable = pl.ok && pl.total != 0ull && variant;
        if (!variant) latch(F.flags, DVC_E_INVALID);  // a root of another game than the context's
        else if (!pl.ok) latch(F.flags, DVC_E_UNSUPPORTED);
        else if (!pl.total) latch(F.flags, DVC_E_INVALID);
        const uint32_t U = g.tmask & ~g.hand(g.cur) & ~g.rev;
        uint32_t slots = 0;
        for (uint32_t q = 0; q < g.np; ++q)
            if (q != g.cur && ((g.alive >> q) & 1u)) slots += __popc(g.hand(q) & ~g.rev);
        // vanilla: the root's one child block holds every plausible set
        tm.root_legal = tm.set_cells ? tm.budget : (int32_t)(slots * __popc(U));
        tm.done = 0;
        tm.next_free = 1;
        tm.used = 1;
        tm.failed = usable ? 0 : 1;
        Node* nodes = F.nodes + tm.node_off;
        Node r;
        r.visits = 0;
        r.wins = 0;
        r.child = -1;
        r.meta = 0u;
        nodes[0] = r;
        F.link[tm.node_off] = -1;
        F.created[tm.node_off] = -1;
        pipe_np[t] = -1;  // no pipeline backprop pending
    }
    for (int32_t c = (int32_t)lane; c < tm.set_cells; c += 32) F.set_slot[tm.set_off + c] = -1;
    __syncwarp();
}

// Every tree, optionally with new roots.
__global__ void forest_init_kernel(ForestDev F, int n, const dvc_state* new_roots, DetPlan* plans,
                                   unsigned long long* tables, uint32_t table_cap, int nplayers, int ntiles,
                                   int32_t* pipe_np) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= n) return;
    if (new_roots && (threadIdx.x & 31u) == 0) const_cast<dvc_state*>(F.roots)[t] = new_roots[t];
    __syncwarp();
    init_tree(F, t, plans, tables, table_cap, nplayers, ntiles, pipe_np);
}

// Selected trees take a new root, budget and stream id (a new search).
__global__ void forest_admit_kernel(ForestDev F, int count, const int32_t* slots, const dvc_state* new_roots,
                                    const int32_t* budgets, const uint32_t* tree_ids, DetPlan* plans,
                                    unsigned long long* tables, uint32_t table_cap, int nplayers, int ntiles,
                                    int32_t* pipe_np) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= count) return;
    const int t = slots[i];
    if ((threadIdx.x & 31u) == 0) {
        const_cast<dvc_state*>(F.roots)[t] = new_roots[i];
        F.meta[t].budget = budgets[i];
        F.meta[t].tree_id = tree_ids[i];
    }
    __syncwarp();
    init_tree(F, t, plans, tables, table_cap, nplayers, ntiles, pipe_np);
}

// Budgets of all trees set to `b` (0 = every tree idle).
__global__ void forest_set_budget_kernel(TreeMeta* meta, int n, int32_t b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) meta[t].budget = b;
}

ForestDev dev_of(dvc_forest* f) {
    ForestDev d;
    d.roots = f->roots;
    d.meta = f->meta;
    d.plans = f->plans;
    d.tables = f->tables;
    d.nodes = f->nodes;
    d.link = f->link;
    d.created = f->created;
    d.ucb = f->ucb;
    d.csl = f->csl;
    d.flags = f->ctx->d_flags;
    d.words = f->no_count ? nullptr : f->d_words;
    d.set_key = f->set_key;
    d.set_slot = f->set_slot;
    return d;
}

SearchParams params_of(const dvc_forest* f) {
    SearchParams sp;
    sp.seed = f->seed;
    sp.c_uct = (float)f->ctx->cfg.c_uct;  // rounded to nearest, as the UCB1 arithmetic is single precision
    sp.d_max = f->ctx->cfg.d_max;
    sp.playouts = f->ctx->cfg.playouts;
    sp.cont_thr = f->ctx->cfg.cont_thr;
    sp.policy = f->ctx->cfg.policy;
    sp.tree_continue = f->ctx->cfg.tree_continue;
    return sp;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

int dvc_create(dvc_ctx** out, const dvc_config* cfg, int device) {
    if (!out || !cfg) return DVC_E_INVALID;
    *out = nullptr;
    if (cfg->nplayers < 2 || cfg->nplayers > 4) return DVC_E_INVALID;
    if (cfg->ntiles != 24 && cfg->ntiles != 26) return DVC_E_INVALID;
    if (cfg->deal < 1 || cfg->nplayers * cfg->deal >= cfg->ntiles) return DVC_E_INVALID;
    if (cfg->max_predraw < 0 || cfg->max_predraw > 24 || cfg->max_revealed < 0) return DVC_E_INVALID;
    if (cfg->d_max < 0 || cfg->d_max > kPathMax - 2 || cfg->playouts < 1 || cfg->playouts > (1 << 20))
        return DVC_E_INVALID;
    if (!(cfg->c_uct >= 0.0)) return DVC_E_INVALID;
    if (cfg->policy != 0 && cfg->policy != 1) return DVC_E_INVALID;
    if (cfg->tree_continue != 0 && cfg->tree_continue != 1) return DVC_E_INVALID;
    if (cfg->vanilla != 0 && cfg->vanilla != 1) return DVC_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DVC_E_CUDA;
    }
    dvc_ctx* c = new (std::nothrow) dvc_ctx();
    if (!c) return DVC_E_OOM;
    c->cfg = *cfg;
    c->device = device;
    c->d_flags = nullptr;
    c->d_ws = nullptr;
    c->ws_cells = 0;
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&c->d_flags, 16) != cudaSuccess ||
        cudaMemset(c->d_flags, 0, 16) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_flags) cudaFree(c->d_flags);
        delete c;
        return DVC_E_CUDA;
    }
    *out = c;
    return DVC_OK;
}

void dvc_destroy(dvc_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    dvc_value_free(c);
    if (c->d_flags) cudaFree(c->d_flags);
    if (c->d_ws) cudaFree(c->d_ws);
    delete c;
}

const char* dvc_last_error(const dvc_ctx* c) { return c ? c->err.c_str() : "null context"; }

int dvc_check(dvc_ctx* c) {
    if (!c) return DVC_E_INVALID;
    if (int rc = set_device(c)) return rc;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "dvc_check");
    int32_t flag = 0;
    e = cudaMemcpy(&flag, c->d_flags, sizeof(flag), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "dvc_check");
    if (flag) {
        cudaMemset(c->d_flags, 0, 16);
        return fail(c, flag, "a kernel latched error " + std::to_string(flag));
    }
    return DVC_OK;
}

int dvc_philox(dvc_ctx* c, int n, const uint32_t* d_ctr, const uint32_t* d_key, uint32_t* d_out, int use_reference,
               void* stream) {
    if (!c) return DVC_E_INVALID;
    if (n < 0) return fail(c, DVC_E_INVALID, "dvc_philox: n < 0");
    if (n == 0) return DVC_OK;
    if (!is_device_ptr(d_ctr, c->device) || !is_device_ptr(d_key, c->device) || !is_device_ptr(d_out, c->device))
        return fail(c, DVC_E_INVALID, "dvc_philox: pointers must be device memory");
    if (int rc = set_device(c)) return rc;
    philox_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, d_ctr, d_key, d_out, use_reference);
    return check_launch(c, "philox_kernel");
}

int dvc_init_states(dvc_ctx* c, uint64_t seed, int n, dvc_state* d_states, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (n < 0) return fail(c, DVC_E_INVALID, "dvc_init_states: n < 0");
    if (n == 0) return DVC_OK;
    if (!is_device_ptr(d_states, c->device)) return fail(c, DVC_E_INVALID, "dvc_init_states: d_states must be device memory");
    if (int rc = set_device(c)) return rc;
    init_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(c->cfg, seed, n, d_states);
    return check_launch(c, "init_kernel");
}

int dvc_determinize(dvc_ctx* c, const dvc_state* d_roots, int n, int observer, uint64_t seed,
                    const uint32_t* d_tree_ids, const uint32_t* d_iter_ids, dvc_state* d_out, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (n < 0 || observer >= c->cfg.nplayers) return fail(c, DVC_E_INVALID, "dvc_determinize: bad n or observer");
    if (n == 0) return DVC_OK;
    if (!is_device_ptr(d_roots, c->device) || !is_device_ptr(d_tree_ids, c->device) || !is_device_ptr(d_iter_ids, c->device) ||
        !is_device_ptr(d_out, c->device))
        return fail(c, DVC_E_INVALID, "dvc_determinize: pointers must be device memory");
    if (ranges_overlap(d_roots, d_out, sizeof(dvc_state) * (size_t)n))
        return fail(c, DVC_E_INVALID, "dvc_determinize: d_out may not overlap d_roots");
    if (int rc = set_device(c)) return rc;
    if (!c->d_ws) {
        const size_t cells = (size_t)kDetChunk * kDetMaxCells;
        if (cudaMalloc(&c->d_ws, cells * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            c->d_ws = nullptr;
            return fail(c, DVC_E_OOM, "dvc_determinize: workspace");
        }
        c->ws_cells = cells;
    }
    for (int base = 0; base < n; base += kDetChunk) {
        const int m = std::min(kDetChunk, n - base);
        determinize_kernel<<<(m + 63) / 64, 64, 0, (cudaStream_t)stream>>>(
            d_roots + base, m, observer, seed, d_tree_ids + base, d_iter_ids + base, d_out + base, c->d_ws,
            c->d_flags);
        if (int rc = check_launch(c, "determinize_kernel")) return rc;
    }
    return DVC_OK;
}

int dvc_rollout_batch(dvc_ctx* c, const dvc_state* d_leaves, int n_leaves, int playouts_per_leaf, uint64_t seed,
                      const uint32_t* d_tree_ids, const uint32_t* d_leaf_ids, int32_t* d_wins, uint64_t* d_words,
                      void* stream) {
    if (!c) return DVC_E_INVALID;
    if (n_leaves < 0 || playouts_per_leaf < 1) return fail(c, DVC_E_INVALID, "dvc_rollout_batch: bad sizes");
    if (n_leaves == 0) return DVC_OK;
    if (!is_device_ptr(d_leaves, c->device) || !is_device_ptr(d_tree_ids, c->device) || !is_device_ptr(d_leaf_ids, c->device) ||
        !is_device_ptr(d_wins, c->device) || (d_words && !is_device_ptr(d_words, c->device)))
        return fail(c, DVC_E_INVALID, "dvc_rollout_batch: pointers must be device memory");
    if (int rc = set_device(c)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_wins, 0, sizeof(int32_t) * 4 * (size_t)n_leaves, st);
    if (e == cudaSuccess && d_words) e = cudaMemsetAsync(d_words, 0, sizeof(uint64_t), st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dvc_rollout_batch memset");
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
    const long long total = (long long)n_leaves * playouts_per_leaf;
    const int block = 256;
    long long blocks = (total + block - 1) / block;
    blocks = std::min<long long>(blocks, (long long)dev_sms * 64);
    if (c->cfg.policy)
        rollout_kernel<true><<<(unsigned)blocks, block, 0, st>>>(d_leaves, n_leaves, playouts_per_leaf, seed,
                                                                 d_tree_ids, d_leaf_ids, c->cfg.cont_thr, d_wins,
                                                                 (unsigned long long*)d_words, c->d_flags);
    else
        rollout_kernel<false><<<(unsigned)blocks, block, 0, st>>>(d_leaves, n_leaves, playouts_per_leaf, seed,
                                                                  d_tree_ids, d_leaf_ids, c->cfg.cont_thr, d_wins,
                                                                  (unsigned long long*)d_words, c->d_flags);
    return check_launch(c, "rollout_kernel");
}

int dvc_play_move(dvc_ctx* c, dvc_state* d_states, int n, const int32_t* d_actions, uint64_t seed,
                  const uint32_t* d_game_ids, uint32_t turn, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (n < 0) return fail(c, DVC_E_INVALID, "dvc_play_move: n < 0");
    if (n == 0) return DVC_OK;
    if (!is_device_ptr(d_states, c->device) || !is_device_ptr(d_actions, c->device) || (d_game_ids && !is_device_ptr(d_game_ids, c->device)))
        return fail(c, DVC_E_INVALID, "dvc_play_move: pointers must be device memory");
    if (int rc = set_device(c)) return rc;
    play_move_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_states, n, d_actions, seed, d_game_ids, turn,
                                                                         c->cfg.tree_continue != 0, c->d_flags);
    return check_launch(c, "play_move_kernel");
}

void dvc_forest_destroy(dvc_forest* f) {
    if (!f) return;
    cudaSetDevice(f->ctx->device);
    if (f->chunk_exec) cudaGraphExecDestroy(f->chunk_exec);
    if (f->value_exec) cudaGraphExecDestroy(f->value_exec);
    dvc_value_rows_free(&f->vrows);
    if (f->cap_stream) cudaStreamDestroy(f->cap_stream);
    for (int k = 0; k < kMaxChains - 1; ++k) {
        if (f->chain_stream[k]) cudaStreamDestroy(f->chain_stream[k]);
        if (f->join_ev[k]) cudaEventDestroy(f->join_ev[k]);
    }
    if (f->fork_ev) cudaEventDestroy(f->fork_ev);
    void* ptrs[] = {f->set_key,   f->set_slot,
                    f->roots,     f->meta,      f->plans,     f->tables,         f->nodes,         f->link,
                    f->created,   f->work,      f->paths,     f->movers,         f->leaves,        f->leaf_tree,
                    f->leaf_iter, f->d_words,   f->export_scratch, f->order,     f->ucb,           f->csl,
                    f->pipe.leaf, f->pipe.path, f->pipe.mover, f->pipe.np,       f->pipe.wins,     f->pipe.step_end,
                    f->pipe.det,  f->pipe.tree0, f->pipe.det_base, f->probs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete f;
}

int dvc_forest_create(dvc_ctx* c, int n, const dvc_state* d_roots, const int32_t* h_budgets,
                      const uint32_t* h_tree_ids, uint64_t seed, dvc_forest** out, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (!out || n < 1 || !h_budgets) return fail(c, DVC_E_INVALID, "dvc_forest_create: bad arguments");
    *out = nullptr;
    if (!is_device_ptr(d_roots, c->device)) return fail(c, DVC_E_INVALID, "dvc_forest_create: d_roots must be device memory");
    for (int i = 0; i < n; ++i)
        if (h_budgets[i] < 0 || h_budgets[i] > (1 << 24))
            return fail(c, DVC_E_INVALID, "dvc_forest_create: budgets must be in 0..2^24");
    if (int rc = set_device(c)) return rc;
    dvc_forest* f = new (std::nothrow) dvc_forest();
    if (!f) return fail(c, DVC_E_OOM, "dvc_forest_create: host allocation");
    f->h_budgets.assign(h_budgets, h_budgets + n);
    f->ctx = c;
    f->n = n;
    f->seed = seed;
    f->table_cap = c->cfg.nplayers == 2 ? kDetMaxCells2p : kDetMaxCells;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<TreeMeta> hm(n);
    long long slots = 0, cells = 0;
    const bool vanilla = c->cfg.vanilla != 0;
    for (int t = 0; t < n; ++t) {
        TreeMeta& m = hm[t];
        std::memset(&m, 0, sizeof(m));
        m.node_off = slots;
        m.table_off = (long long)t * f->table_cap;
        // vanilla: the root's block holds up to one plausible set per iteration
        m.cap = 1 + (vanilla ? f->h_budgets[t] : kRootReserve) + 4 * f->h_budgets[t];
        m.budget = f->h_budgets[t];
        m.tree_id = h_tree_ids ? h_tree_ids[t] : (uint32_t)t;
        m.set_off = cells;
        m.set_cells = vanilla ? 2 * f->h_budgets[t] : 0;
        slots += m.cap;
        cells += m.set_cells;
    }
    f->total_slots = slots;
    // Longest budget first, each tree to the least-loaded CTA that has a free
    // slot (CTAs hold trees_per_cta trees): balances uneven forests.
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    // enough trees to fill the GPU: the pipeline; small forests: the fused
    // lockstep kernel
    f->engine = n > 4 * std::max(sms, 1) ? 2 : 1;
    default_shape(n, sms, f->engine, c->cfg.playouts, f->trees_per_cta, f->warps_per_cta, f->chains);
    std::vector<int32_t> order(n);
    {
        const int T = f->trees_per_cta;
        const int nc = (n + T - 1) / T;
        std::vector<int> idx(n);
        for (int i = 0; i < n; ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return f->h_budgets[a] > f->h_budgets[b]; });
        bool even = true;
        for (int t = 1; t < n; ++t) even &= f->h_budgets[t] == f->h_budgets[0];
        std::vector<long long> load(nc, 0);
        std::vector<int> fill(nc, 0);
        std::vector<int> capc(nc, T);
        capc[nc - 1] = n - (nc - 1) * T;
        // min-heap of (load, cta)
        std::vector<std::pair<long long, int>> heap;
        for (int k = 0; k < nc; ++k) heap.push_back({0, k});
        auto cmp = [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) { return a > b; };
        std::make_heap(heap.begin(), heap.end(), cmp);
        for (int i : idx) {
            if (even) break;  // equal budgets: keep trees in index order (slot s -> CTA s / T)
            std::pop_heap(heap.begin(), heap.end(), cmp);
            auto [ld, k] = heap.back();
            heap.pop_back();
            order[k * T + fill[k]] = i;
            fill[k]++;
            load[k] = ld + f->h_budgets[i];
            if (fill[k] < capc[k]) {
                heap.push_back({load[k], k});
                std::push_heap(heap.begin(), heap.end(), cmp);
            }
        }
        if (even)
            for (int i = 0; i < n; ++i) order[i] = i;
    }
    auto alloc = [&](void** p, size_t bytes) {
        if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        return true;
    };
    const bool ok =
        alloc((void**)&f->roots, sizeof(dvc_state) * n) && alloc((void**)&f->meta, sizeof(TreeMeta) * n) &&
        alloc((void**)&f->plans, sizeof(DetPlan) * n) && alloc((void**)&f->work, sizeof(Descent) * n) &&
        alloc((void**)&f->paths, sizeof(int32_t) * kPathMax * n) && alloc((void**)&f->movers, kPathMax * (size_t)n) &&
        alloc((void**)&f->leaves, sizeof(dvc_state) * n) && alloc((void**)&f->leaf_tree, sizeof(uint32_t) * n) &&
        alloc((void**)&f->leaf_iter, sizeof(uint32_t) * n) && alloc((void**)&f->d_words, 2 * sizeof(unsigned long long)) &&
        alloc((void**)&f->tables, sizeof(unsigned long long) * (size_t)f->table_cap * n) &&
        alloc((void**)&f->nodes, sizeof(Node) * (size_t)slots) && alloc((void**)&f->link, sizeof(int32_t) * (size_t)slots) &&
        alloc((void**)&f->created, sizeof(int32_t) * (size_t)slots) && alloc((void**)&f->order, sizeof(int32_t) * n) &&
        alloc((void**)&f->ucb, sizeof(float2) * (size_t)slots) && alloc((void**)&f->csl, sizeof(float) * (size_t)slots) &&
        alloc((void**)&f->pipe.leaf, sizeof(dvc_state) * n) && alloc((void**)&f->pipe.path, sizeof(int32_t) * kPathMax * n) &&
        alloc((void**)&f->pipe.mover, (size_t)kPathMax * n) && alloc((void**)&f->pipe.np, sizeof(int32_t) * n) &&
        alloc((void**)&f->pipe.wins, sizeof(int32_t) * 4 * n) && alloc((void**)&f->pipe.step_end, sizeof(int32_t) * n) &&
        alloc((void**)&f->pipe.det, sizeof(dvc_state) * kDetAhead * (size_t)n) &&
        alloc((void**)&f->pipe.tree0, sizeof(uint4) * kDetAhead * (size_t)n) &&
        alloc((void**)&f->pipe.det_base, sizeof(int32_t) * n) &&
        (!vanilla || (alloc((void**)&f->set_key, sizeof(uint4) * (size_t)cells) &&
                      alloc((void**)&f->set_slot, sizeof(int32_t) * (size_t)cells)));
    if (!ok) {
        dvc_forest_destroy(f);
        return fail(c, DVC_E_OOM, "dvc_forest_create: device allocation of " + std::to_string(slots) + " node slots");
    }
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    cudaError_t e = cudaMemcpyAsync(f->meta, hm.data(), sizeof(TreeMeta) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->roots, d_roots, sizeof(dvc_state) * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_words, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->pipe.det_base, 0xC0, sizeof(int32_t) * n, st);  // none ahead
    f->pipe.flags = c->d_flags;
    if (e != cudaSuccess) {
        dvc_forest_destroy(f);
        return cuda_fail(c, e, "dvc_forest_create copy");
    }
    forest_init_kernel<<<(n * 32 + 127) / 128, 128, 0, st>>>(dev_of(f), n, nullptr, f->plans, f->tables, f->table_cap,
                                                            c->cfg.nplayers, c->cfg.ntiles, f->pipe.np);
    if (int rc = check_launch(c, "forest_init_kernel")) {
        dvc_forest_destroy(f);
        return rc;
    }
    bool sok = cudaStreamCreateWithFlags(&f->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&f->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kMaxChains - 1 && sok; ++k)
        sok = cudaStreamCreateWithFlags(&f->chain_stream[k], cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&f->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!sok) {
        cudaGetLastError();
        dvc_forest_destroy(f);
        return fail(c, DVC_E_CUDA, "dvc_forest_create: streams");
    }
    *out = f;
    return DVC_OK;
}

int dvc_forest_reset(dvc_forest* f, const dvc_state* d_roots, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (d_roots && !is_device_ptr(d_roots, f->ctx->device))
        return fail(f->ctx, DVC_E_INVALID, "dvc_forest_reset: d_roots must be device memory");
    if (int rc = set_device(f->ctx)) return rc;
    f->active_prefix = 0;  // every tree has its budget again
    forest_init_kernel<<<(f->n * 32 + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        dev_of(f), f->n, d_roots, f->plans, f->tables, f->table_cap, f->ctx->cfg.nplayers, f->ctx->cfg.ntiles,
        f->pipe.np);
    return check_launch(f->ctx, "forest_init_kernel");
}

}  // extern "C"

namespace {

// The default tree order for CTAs of T trees: longest budget first, each to
// the least-loaded CTA (equal budgets keep index order); host work, one copy.
// Clears a caller's active prefix (it referred to the order replaced here).
int set_default_order(dvc_forest* f, int T) {
    std::vector<int32_t> order(f->n);
    const int nc = (f->n + T - 1) / T;
    std::vector<int> idx(f->n);
    for (int i = 0; i < f->n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return f->h_budgets[a] > f->h_budgets[b]; });
    std::vector<std::pair<long long, int>> heap;
    std::vector<int> fill(nc, 0), capc(nc, T);
    capc[nc - 1] = f->n - (nc - 1) * T;
    for (int k = 0; k < nc; ++k) heap.push_back({0, k});
    auto cmp = [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) { return a > b; };
    std::make_heap(heap.begin(), heap.end(), cmp);
    bool even = true;
    for (int t = 1; t < f->n; ++t) even &= f->h_budgets[t] == f->h_budgets[0];
    for (int i : idx) {
        if (even) break;  // equal budgets: index order
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto [ld, k] = heap.back();
        heap.pop_back();
        order[k * T + fill[k]++] = i;
        if (fill[k] < capc[k]) {
            heap.push_back({ld + f->h_budgets[i], k});
            std::push_heap(heap.begin(), heap.end(), cmp);
        }
    }
    if (even)
        for (int i = 0; i < f->n; ++i) order[i] = i;
    if (int rc = set_device(f->ctx)) return rc;
    const cudaError_t e = cudaMemcpy(f->order, order.data(), sizeof(int32_t) * f->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(f->ctx, e, "forest order");
    f->active_prefix = 0;
    return DVC_OK;
}

int launch_fused(dvc_forest* f, int n_iterations, cudaStream_t st) {
    dvc_ctx* c = f->ctx;
    const int T = f->trees_per_cta;
    const int W = std::max(1, std::min(32, f->warps_per_cta ? f->warps_per_cta : std::min(T, 16)));
    const int n_run = f->active_prefix > 0 ? std::min(f->n, f->active_prefix) : f->n;
    const int grid = (n_run + T - 1) / T;
    const PoolLayout L(T, W);
    const int threads = 32 * W;
    const bool fast2 = c->cfg.nplayers == 2 && c->cfg.ntiles == 24;
    cudaError_t e;
#define DVC_LAUNCH_POOL(MT, F2, ORD)                                                                              \
    do {                                                                                                          \
        e = cudaFuncSetAttribute(mcts_pool_kernel<MT, F2, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                 (int)L.bytes);                                                                   \
        if (e == cudaSuccess)                                                                                     \
            mcts_pool_kernel<MT, F2, ORD><<<grid, threads, L.bytes, st>>>(dev_of(f), params_of(f), n_iterations,  \
                                                                          f->order, f->n, T, f->pipe.det,         \
                                                                          f->pipe.tree0);                         \
    } while (0)
    if (c->cfg.policy && threads <= 512) {  // ordering-aware playouts
        if (fast2) DVC_LAUNCH_POOL(512, true, true);
        else DVC_LAUNCH_POOL(512, false, true);
    } else if (c->cfg.policy) {
        if (fast2) DVC_LAUNCH_POOL(1024, true, true);
        else DVC_LAUNCH_POOL(1024, false, true);
    } else if (threads <= 512) {
        if (fast2) DVC_LAUNCH_POOL(512, true, false);
        else DVC_LAUNCH_POOL(512, false, false);
    } else if (threads <= 768) {
        if (fast2) DVC_LAUNCH_POOL(768, true, false);
        else DVC_LAUNCH_POOL(768, false, false);
    } else {
        if (fast2) DVC_LAUNCH_POOL(1024, true, false);
        else DVC_LAUNCH_POOL(1024, false, false);
    }
#undef DVC_LAUNCH_POOL
    if (e != cudaSuccess) return cuda_fail(c, e, "mcts_pool_kernel attributes");
    return check_launch(c, "mcts_pool_kernel");
}

int pipe_rollout_threads(const dvc_forest* f) { return 32 * (f->warps_per_cta ? f->warps_per_cta : 32); }

// One pipeline iteration of the trees of CTAs [b0, b1): (pending backprop +)
// select, then rollouts.
int enqueue_pipe_iteration(dvc_forest* f, int b0, int b1, cudaStream_t st) {
    dvc_ctx* c = f->ctx;
    const ForestDev fd = dev_of(f);
    const SearchParams sp = params_of(f);
    const int n = f->n, L = f->trees_per_cta;
    const int i0 = std::min(n, b0 * L), i1 = std::min(n, b1 * L);
    if (i1 <= i0) return DVC_OK;
    if (c->cfg.vanilla)
        pipe_select_kernel<true><<<((i1 - i0) * 32 + 127) / 128, 128, 0, st>>>(fd, sp, i0, i1, f->order, f->pipe);
    else
        pipe_select_kernel<false><<<((i1 - i0) * 32 + 127) / 128, 128, 0, st>>>(fd, sp, i0, i1, f->order, f->pipe);
    const int threads = pipe_rollout_threads(f);
    const bool fast2 = c->cfg.nplayers == 2 && c->cfg.ntiles == 24;
    // may-stop leaves possible: the full tree, or leaves that can be the root itself
    const bool pend = c->cfg.tree_continue || c->cfg.d_max == 0 || c->cfg.vanilla;
    const uint32_t smem = pipe_rollout_smem(L, threads);
    unsigned long long* words = f->no_count ? nullptr : f->d_words;
    if (fast2 && !sp.policy && !pend && f->cmp_receivers > 0 && f->cmp_receivers < threads / 32)
        pipe_rollout_compact_kernel<<<b1 - b0, threads, pipe_compact_smem(L, threads, f->cmp_receivers), st>>>(
            sp, n, L, b0, f->order, f->meta, f->pipe, words, f->cmp_receivers, f->cmp_donate_at);
    else if (fast2 && !sp.policy && !pend && f->no_count)
        pipe_rollout_kernel<true, false, false, false><<<b1 - b0, threads, smem, st>>>(sp, n, L, b0, f->order,
                                                                                      f->meta, f->pipe, nullptr);
    else if (fast2 && !sp.policy && !pend)
        pipe_rollout_kernel<true, false, false><<<b1 - b0, threads, smem, st>>>(sp, n, L, b0, f->order, f->meta,
                                                                               f->pipe, words);
    else if (fast2 && !sp.policy)
        pipe_rollout_kernel<true, false, true><<<b1 - b0, threads, smem, st>>>(sp, n, L, b0, f->order, f->meta,
                                                                              f->pipe, words);
    else if (fast2)
        pipe_rollout_kernel<true, true><<<b1 - b0, threads, smem, st>>>(sp, n, L, b0, f->order, f->meta, f->pipe,
                                                                       words);
    else if (!sp.policy)
        pipe_rollout_kernel<false, false><<<b1 - b0, threads, smem, st>>>(sp, n, L, b0, f->order, f->meta, f->pipe,
                                                                         words);
    else
        pipe_rollout_kernel<false, true><<<b1 - b0, threads, smem, st>>>(sp, n, L, b0, f->order, f->meta, f->pipe,
                                                                        words);
    return check_launch(c, "pipeline kernels");
}

// Sample the next `count` determinizations of the trees of CTAs [b0, b1) ahead.
int enqueue_pipe_det(dvc_forest* f, int b0, int b1, int count, cudaStream_t st) {
    const int n = f->n, L = f->trees_per_cta;
    const int i0 = std::min(n, b0 * L), i1 = std::min(n, b1 * L);
    if (i1 <= i0 || count <= 0) return DVC_OK;
    const long long threads = (long long)(i1 - i0) * count;
    pipe_det_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(dev_of(f), params_of(f), i0, i1, f->order,
                                                                       f->pipe, count);
    return check_launch(f->ctx, "pipe_det_kernel");
}

// Outside a pipeline step no tree has determinizations sampled ahead.
int clear_pipe_det(dvc_forest* f, cudaStream_t st) {
    // 0xC0C0C0C0 is below -2^29: no iteration lies within kDetAhead of it
    const cudaError_t e = cudaMemsetAsync(f->pipe.det_base, 0xC0, sizeof(int32_t) * f->n, st);
    return e == cudaSuccess ? DVC_OK : cuda_fail(f->ctx, e, "pipeline determinization buffer");
}

constexpr int kChunkIters = 64;
static_assert(kChunkIters <= kDetAhead, "a chunk's determinizations are sampled at its start");

// CTA range of chain k when the grid is split into `chains` independent chains.
void chain_range(const dvc_forest* f, int k, int chains, int& b0, int& b1) {
    const int grid = (f->n + f->trees_per_cta - 1) / f->trees_per_cta;
    b0 = (int)((long long)grid * k / chains);
    b1 = (int)((long long)grid * (k + 1) / chains);
}

// Capture kChunkIters iterations into *exec: `chains` independent chains on
// their own streams (forked from and joined to the capture stream), so one
// chain's tree walks overlap another chain's leaf scoring on the same SMs.
// begin(k, stream) runs once per chain, then step(k, stream) per iteration.
template <class Begin, class Step>
int capture_chains(dvc_forest* f, int chains, cudaGraphExec_t* exec, Begin begin, Step step) {
    dvc_ctx* c = f->ctx;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(f->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "pipeline capture");
    int rc = DVC_OK;
    cudaStream_t ss[kMaxChains] = {f->cap_stream};
    for (int k = 1; k < kMaxChains; ++k) ss[k] = f->chain_stream[k - 1];
    if (chains > 1) {
        e = cudaEventRecord(f->fork_ev, f->cap_stream);
        for (int k = 1; k < chains && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(ss[k], f->fork_ev, 0);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "pipeline fork");
    }
    for (int k = 0; k < chains && rc == DVC_OK; ++k) rc = begin(k, ss[k]);
    for (int it = 0; it < kChunkIters && rc == DVC_OK; ++it)
        for (int k = 0; k < chains && rc == DVC_OK; ++k) rc = step(k, ss[k]);
    if (rc == DVC_OK && chains > 1) {
        for (int k = 1; k < chains && e == cudaSuccess; ++k) {
            e = cudaEventRecord(f->join_ev[k - 1], ss[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(f->cap_stream, f->join_ev[k - 1], 0);
        }
        if (e != cudaSuccess) rc = cuda_fail(c, e, "pipeline join");
    }
    e = cudaStreamEndCapture(f->cap_stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "pipeline capture end");
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return cuda_fail(c, e, "pipeline graph");
    }
    return DVC_OK;
}

// Rollout mode: the forest's rollout CTAs split into chains.
int capture_chunk(dvc_forest* f) {
    const int chains = std::max(1, std::min(kMaxChains, f->chains));
    return capture_chains(
        f, chains, &f->chunk_exec,
        [&](int k, cudaStream_t s) {
            int b0, b1;
            chain_range(f, k, chains, b0, b1);
            return enqueue_pipe_det(f, b0, b1, kChunkIters, s);
        },
        [&](int k, cudaStream_t s) {
            int b0, b1;
            chain_range(f, k, chains, b0, b1);
            return enqueue_pipe_iteration(f, b0, b1, s);
        });
}

int launch_pipeline(dvc_forest* f, int n_iterations, cudaStream_t st) {
    dvc_ctx* c = f->ctx;
    {
        const int threads = pipe_rollout_threads(f);
        const int sm = (int)pipe_rollout_smem(f->trees_per_cta, threads);
        cudaError_t e = cudaSuccess;
        // several rollout CTAs per SM need the largest shared-memory carveout
        for (auto k : {pipe_rollout_kernel<true, false, false>, pipe_rollout_kernel<true, false, false, false>,
                       pipe_rollout_kernel<true, false, true>, pipe_rollout_kernel<true, true, true>,
                       pipe_rollout_kernel<false, false, true>, pipe_rollout_kernel<false, true, true>}) {
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
        }
        if (e == cudaSuccess && f->cmp_receivers > 0) {
            const int smc = (int)pipe_compact_smem(f->trees_per_cta, threads, f->cmp_receivers);
            e = cudaFuncSetAttribute(pipe_rollout_compact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smc);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(pipe_rollout_compact_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "pipeline attributes");
    }
    if (int rc = clear_pipe_det(f, st)) return rc;
    pipe_begin_kernel<<<(f->n + 127) / 128, 128, 0, st>>>(dev_of(f), f->n, n_iterations, f->pipe.step_end);
    if (int rc = check_launch(c, "pipe_begin_kernel")) return rc;
    int left = n_iterations;
    if (left >= kChunkIters) {
        if (!f->chunk_exec)
            if (int rc = capture_chunk(f)) return rc;
        while (left >= kChunkIters) {
            const cudaError_t e = cudaGraphLaunch(f->chunk_exec, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "pipeline graph launch");
            left -= kChunkIters;
        }
    }
    const int grid = (f->n + f->trees_per_cta - 1) / f->trees_per_cta;
    if (int rc = enqueue_pipe_det(f, 0, grid, left, st)) return rc;
    for (; left > 0; --left)
        if (int rc = enqueue_pipe_iteration(f, 0, grid, st)) return rc;
    pipe_backprop_kernel<<<(f->n * 32 + 127) / 128, 128, 0, st>>>(dev_of(f), params_of(f), f->n, f->pipe);
    return check_launch(c, "pipe_backprop_kernel");
}

// Value mode.  Trees t0 .. t1-1 of chain k (index order; each chain's leaves
// are contiguous so the network reads them in place) and the first row of the
// chain's activation slice.
void value_chain(const dvc_forest* f, int k, int chains, int& t0, int& t1, int& row0) {
    row0 = 0;
    for (int j = 0; j <= k; ++j) {
        t0 = (int)((long long)f->n * j / chains);
        t1 = (int)((long long)f->n * (j + 1) / chains);
        if (j < k) row0 += (t1 - t0 + 127) / 128 * 128;
    }
}

int value_chains(const dvc_forest* f) { return std::max(1, std::min({kValueChains, f->chains, f->n / 128})); }

// One value-mode iteration of chain k: (pending backprop +) select, the
// network over the chain's leaves, credit.
int enqueue_value_iteration(dvc_forest* f, int k, int chains, cudaStream_t st) {
    dvc_ctx* c = f->ctx;
    int t0, t1, row0;
    value_chain(f, k, chains, t0, t1, row0);
    if (t1 <= t0) return DVC_OK;
    if (c->cfg.vanilla)
        pipe_select_kernel<true><<<((t1 - t0) * 32 + 127) / 128, 128, 0, st>>>(dev_of(f), params_of(f), t0, t1,
                                                                                nullptr, f->pipe);
    else
        pipe_select_kernel<false><<<((t1 - t0) * 32 + 127) / 128, 128, 0, st>>>(dev_of(f), params_of(f), t0, t1,
                                                                                 nullptr, f->pipe);
    if (int rc = check_launch(c, "pipe_select_kernel")) return rc;
    if (int rc = dvc_value_forward_rows(c, f->pipe.leaf + t0, t1 - t0, &f->vrows, row0, f->probs + 4 * (size_t)t0, st))
        return rc;
    pipe_value_wins_kernel<<<(t1 - t0 + 127) / 128, 128, 0, st>>>(t0, t1, f->pipe, f->probs, f->ctx->cfg.playouts);
    return check_launch(c, "pipe_value_wins_kernel");
}

int enqueue_value_det(dvc_forest* f, int k, int chains, int count, cudaStream_t st) {
    int t0, t1, row0;
    value_chain(f, k, chains, t0, t1, row0);
    if (t1 <= t0 || count <= 0) return DVC_OK;
    const long long threads = (long long)(t1 - t0) * count;
    pipe_det_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(dev_of(f), params_of(f), t0, t1, nullptr,
                                                                       f->pipe, count);
    return check_launch(f->ctx, "pipe_det_kernel");
}

// Value mode: the same chained, graph-captured pipeline as rollout mode, the
// rollout launch replaced by the network over each chain's leaves.
int launch_value_pipeline(dvc_forest* f, int n_iterations, cudaStream_t st) {
    dvc_ctx* c = f->ctx;
    if (!f->probs) {
        if (cudaMalloc(&f->probs, sizeof(float) * 4 * (size_t)f->n) != cudaSuccess) {
            cudaGetLastError();
            f->probs = nullptr;
            return fail(c, DVC_E_OOM, "dvc_mcts_step: value buffer");
        }
    }
    const int chains = value_chains(f);
    int t0, t1, rows;
    value_chain(f, chains - 1, chains, t0, t1, rows);
    rows += (t1 - t0 + 127) / 128 * 128;
    if (f->vrows.rows < rows) {
        if (f->value_exec) cudaGraphExecDestroy(f->value_exec);
        f->value_exec = nullptr;
        if (int rc = dvc_value_rows_alloc(c, &f->vrows, rows)) return rc;
    }
    if (int rc = dvc_value_prepare(c)) return rc;
    if (int rc = clear_pipe_det(f, st)) return rc;
    pipe_begin_kernel<<<(f->n + 127) / 128, 128, 0, st>>>(dev_of(f), f->n, n_iterations, f->pipe.step_end);
    if (int rc = check_launch(c, "pipe_begin_kernel")) return rc;
    int left = n_iterations;
    if (left >= kChunkIters) {
        if (!f->value_exec) {
            const int rc = capture_chains(
                f, chains, &f->value_exec,
                [&](int k, cudaStream_t s) { return enqueue_value_det(f, k, chains, kChunkIters, s); },
                [&](int k, cudaStream_t s) { return enqueue_value_iteration(f, k, chains, s); });
            if (rc) return rc;
        }
        while (left >= kChunkIters) {
            const cudaError_t e = cudaGraphLaunch(f->value_exec, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "value pipeline graph launch");
            left -= kChunkIters;
        }
    }
    for (int k = 0; k < chains; ++k)
        if (int rc = enqueue_value_det(f, k, chains, left, st)) return rc;
    for (; left > 0; --left)
        for (int k = 0; k < chains; ++k)
            if (int rc = enqueue_value_iteration(f, k, chains, st)) return rc;
    pipe_backprop_kernel<<<(f->n * 32 + 127) / 128, 128, 0, st>>>(dev_of(f), params_of(f), f->n, f->pipe);
    return check_launch(c, "pipe_backprop_kernel");
}

}  // namespace

extern "C" {

int dvc_mcts_step(dvc_forest* f, int n_iterations, int mode, void* stream) {
    if (!f) return DVC_E_INVALID;
    dvc_ctx* c = f->ctx;
    if (n_iterations < 0) return fail(c, DVC_E_INVALID, "dvc_mcts_step: n_iterations < 0");
    if (mode != DVC_MODE_ROLLOUT && mode != DVC_MODE_VALUE) return fail(c, DVC_E_INVALID, "dvc_mcts_step: bad mode");
    if (mode == DVC_MODE_VALUE && !c->vnet) return fail(c, DVC_E_INVALID, "dvc_mcts_step: value network not initialised");
    if (n_iterations == 0) return DVC_OK;
    if (int rc = set_device(c)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == DVC_MODE_VALUE) return launch_value_pipeline(f, n_iterations, st);
    return f->engine == 2 ? launch_pipeline(f, n_iterations, st) : launch_fused(f, n_iterations, st);
}

int dvc_forest_tune(dvc_forest* f, int engine, int trees_per_cta, int warps_per_cta, int chains) {
    if (!f) return DVC_E_INVALID;
    if (engine < 0 || engine > 2 || trees_per_cta < 0 || trees_per_cta > 64 || warps_per_cta < 0 ||
        warps_per_cta > 32 || chains < 0 || chains > kMaxChains)
        return fail(f->ctx, DVC_E_INVALID,
                    "dvc_forest_tune: engine 0..2, trees_per_cta 0..64, warps_per_cta 0..32, chains 0..32");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->ctx->device);
    const int eng = engine ? engine : f->engine;
    int dT, dW, dC;
    default_shape(f->n, sms, eng, f->ctx->cfg.playouts, dT, dW, dC);
    const int T = trees_per_cta ? trees_per_cta : dT;
    const int W = warps_per_cta ? warps_per_cta : (trees_per_cta && eng == 1 ? std::min(T, 16) : dW);
    const int oldT = f->trees_per_cta, oldW = f->warps_per_cta, oldC = f->chains;
    const PoolLayout L(T, W);
    if (L.bytes > 200 * 1024) return fail(f->ctx, DVC_E_UNSUPPORTED, "dvc_forest_tune: CTA state exceeds shared memory");
    if (T != f->trees_per_cta) {
        if (int rc = set_default_order(f, T)) return rc;
        f->trees_per_cta = T;
    }
    f->engine = eng;
    const int ch = chains ? chains : dC;
    if (W != oldW || T != oldT || ch != oldC) {
        // the captured pipeline graphs hold the old launch shape
        if (f->chunk_exec) cudaGraphExecDestroy(f->chunk_exec);
        if (f->value_exec) cudaGraphExecDestroy(f->value_exec);
        f->chunk_exec = f->value_exec = nullptr;
    }
    f->warps_per_cta = W;
    f->chains = ch;
    return DVC_OK;
}

int dvc_forest_order(dvc_forest* f, const int32_t* h_order, int n_active) {
    if (!f) return DVC_E_INVALID;
    if (!h_order) {  // back to the default order of the current shape
        if (n_active != 0) return fail(f->ctx, DVC_E_INVALID, "dvc_forest_order: the default order runs every tree");
        if (int rc = set_device(f->ctx)) return rc;
        return set_default_order(f, f->trees_per_cta > 0 ? f->trees_per_cta : 1);
    }
    if (n_active < 0 || n_active > f->n) return fail(f->ctx, DVC_E_INVALID, "dvc_forest_order: 0 <= n_active <= trees");
    std::vector<char> seen(f->n, 0);
    for (int i = 0; i < f->n; ++i) {
        const int32_t t = h_order[i];
        if (t < 0 || t >= f->n || seen[t])
            return fail(f->ctx, DVC_E_INVALID, "dvc_forest_order: h_order must be a permutation of the trees");
        seen[t] = 1;
    }
    if (int rc = set_device(f->ctx)) return rc;
    const cudaError_t e = cudaMemcpy(f->order, h_order, sizeof(int32_t) * f->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(f->ctx, e, "dvc_forest_order");
    f->active_prefix = n_active;
    return DVC_OK;
}

int dvc_mcts_select(dvc_forest* f, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (int rc = set_device(f->ctx)) return rc;
    mcts_select_kernel<<<(f->n * 32 + 127) / 128, 128, 0, (cudaStream_t)stream>>>(dev_of(f), params_of(f), f->n,
                                                                                  f->work, f->paths, f->movers);
    return check_launch(f->ctx, "mcts_select_kernel");
}

int dvc_mcts_expand(dvc_forest* f, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (int rc = set_device(f->ctx)) return rc;
    mcts_expand_kernel<<<(f->n * 32 + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        dev_of(f), f->n, f->work, f->paths, f->movers, f->leaves, f->leaf_tree, f->leaf_iter,
        f->ctx->cfg.tree_continue != 0);
    return check_launch(f->ctx, "mcts_expand_kernel");
}

int dvc_mcts_backprop(dvc_forest* f, const int32_t* d_wins, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (!is_device_ptr(d_wins, f->ctx->device)) return fail(f->ctx, DVC_E_INVALID, "dvc_mcts_backprop: d_wins must be device memory");
    if (int rc = set_device(f->ctx)) return rc;
    mcts_backprop_kernel<<<(f->n * 32 + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        dev_of(f), params_of(f), f->n, f->work, f->paths, f->movers, d_wins);
    return check_launch(f->ctx, "mcts_backprop_kernel");
}

int dvc_forest_counters(dvc_forest* f, uint64_t* d_out, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (!is_device_ptr(d_out, f->ctx->device)) return fail(f->ctx, DVC_E_INVALID, "dvc_forest_counters: d_out must be device memory");
    if (int rc = set_device(f->ctx)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_out, f->d_words, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_words, 0, sizeof(uint64_t), st);
    if (e != cudaSuccess) return cuda_fail(f->ctx, e, "dvc_forest_counters");
    return DVC_OK;
}

int dvc_forest_compaction(dvc_forest* f, int receivers, int donate_at) {
    if (!f) return DVC_E_INVALID;
    const int warps = pipe_rollout_threads(f) / 32;
    if (receivers < 0 || (receivers > 0 && (receivers >= warps || donate_at < 1 || donate_at > 31)))
        return fail(f->ctx, DVC_E_INVALID, "dvc_forest_compaction: 0 <= receivers < warps per rollout CTA, 1 <= donate_at <= 31");
    if (receivers != f->cmp_receivers || donate_at != f->cmp_donate_at) {
        if (f->chunk_exec) cudaGraphExecDestroy(f->chunk_exec);  // recaptured with the other kernel
        f->chunk_exec = nullptr;
    }
    f->cmp_receivers = receivers;
    f->cmp_donate_at = receivers ? donate_at : 0;
    return DVC_OK;
}

int dvc_forest_count_work(dvc_forest* f, int on) {
    if (!f) return DVC_E_INVALID;
    const int no = on ? 0 : 1;
    if (no != f->no_count) {  // the captured pipeline graphs hold the other kernels
        if (f->chunk_exec) cudaGraphExecDestroy(f->chunk_exec);
        if (f->value_exec) cudaGraphExecDestroy(f->value_exec);
        f->chunk_exec = f->value_exec = nullptr;
    }
    f->no_count = no;
    return DVC_OK;
}

int dvc_forest_work(dvc_forest* f, uint64_t* d_out, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (!is_device_ptr(d_out, f->ctx->device)) return fail(f->ctx, DVC_E_INVALID, "dvc_forest_work: d_out must be device memory");
    if (int rc = set_device(f->ctx)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_out, f->d_words, 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_words, 0, 2 * sizeof(uint64_t), st);
    if (e != cudaSuccess) return cuda_fail(f->ctx, e, "dvc_forest_work");
    return DVC_OK;
}

int dvc_forest_leaves(dvc_forest* f, dvc_state** d_leaves, uint32_t** d_tree_ids, uint32_t** d_leaf_ids) {
    if (!f || !d_leaves || !d_tree_ids || !d_leaf_ids) return DVC_E_INVALID;
    *d_leaves = f->leaves;
    *d_tree_ids = f->leaf_tree;
    *d_leaf_ids = f->leaf_iter;
    return DVC_OK;
}

int dvc_root_stats(dvc_forest* f, int32_t* d_out, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (!is_device_ptr(d_out, f->ctx->device)) return fail(f->ctx, DVC_E_INVALID, "dvc_root_stats: d_out must be device memory");
    if (int rc = set_device(f->ctx)) return rc;
    if (f->ctx->cfg.vanilla) {
        root_stats_vanilla_kernel<<<f->n, 256, 0, (cudaStream_t)stream>>>(dev_of(f), f->n, d_out);
        return check_launch(f->ctx, "root_stats_vanilla_kernel");
    }
    root_stats_kernel<<<(f->n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(dev_of(f), f->n, d_out);
    return check_launch(f->ctx, "root_stats_kernel");
}

int dvc_root_merge(dvc_forest* f, int K, int32_t* d_out, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (K < 1 || f->n % K) return fail(f->ctx, DVC_E_INVALID, "dvc_root_merge: K must divide the number of trees");
    long long maxb = 0;
    for (int t = 0; t < f->n; ++t) maxb = std::max<long long>(maxb, f->h_budgets[t]);
    if ((long long)K * maxb * f->ctx->cfg.playouts >= (1LL << 31))
        return fail(f->ctx, DVC_E_UNSUPPORTED, "dvc_root_merge: K x budget x playouts must stay below 2^31");
    if (!is_device_ptr(d_out, f->ctx->device)) return fail(f->ctx, DVC_E_INVALID, "dvc_root_merge: d_out must be device memory");
    if (int rc = set_device(f->ctx)) return rc;
    root_merge_kernel<<<f->n / K, 256, 0, (cudaStream_t)stream>>>(dev_of(f), K, f->n / K, f->ctx->cfg.vanilla ? 1 : 0,
                                                                   d_out);
    return check_launch(f->ctx, "root_merge_kernel");
}

int dvc_tree_export(dvc_forest* f, int tree, int32_t* d_out, void* stream) {
    if (!f) return DVC_E_INVALID;
    if (tree < 0 || tree >= f->n) return fail(f->ctx, DVC_E_INVALID, "dvc_tree_export: tree out of range");
    if (!is_device_ptr(d_out, f->ctx->device)) return fail(f->ctx, DVC_E_INVALID, "dvc_tree_export: d_out must be device memory");
    if (int rc = set_device(f->ctx)) return rc;
    const int32_t budget = f->h_budgets[tree];
    if (budget > f->export_cap) {
        if (f->export_scratch) cudaFree(f->export_scratch);
        f->export_scratch = nullptr;
        f->export_cap = 0;
        if (cudaMalloc(&f->export_scratch, sizeof(int32_t) * (size_t)std::max(budget, 1)) != cudaSuccess) {
            cudaGetLastError();
            f->export_scratch = nullptr;
            return fail(f->ctx, DVC_E_OOM, "dvc_tree_export: scratch");
        }
        f->export_cap = budget;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t rows = budget + 1;
    cudaError_t e = cudaMemsetAsync(d_out, 0xFF, sizeof(int32_t) * 4 * (size_t)rows, st);
    if (e == cudaSuccess && budget > 0)
        e = cudaMemsetAsync(f->export_scratch, 0, sizeof(int32_t) * (size_t)budget, st);
    if (e != cudaSuccess) return cuda_fail(f->ctx, e, "dvc_tree_export memset");
    const ForestDev fd = dev_of(f);
    export_flag_kernel<<<64, 256, 0, st>>>(fd, tree, f->export_scratch);
    export_scan_kernel<<<1, 1, 0, st>>>(budget, f->export_scratch);
    export_rows_kernel<<<64, 256, 0, st>>>(fd, tree, f->export_scratch, rows, d_out);
    return check_launch(f->ctx, "export kernels");
}

}  // extern "C"

// ---------------------------------------------------------------- serving

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerQuery {
    dvc_state root;
    int32_t budget;
    int32_t lane;  // the (context, mode) lane that searches it
    uint64_t id;
    double t_submit;
};

struct ServerSlot {
    bool busy = false;
    ServerQuery q;
};

// One game variant (a context) in one leaf mode: a forest whose trees are
// the search slots, its own stream (so the lanes' searches overlap on the
// device), admission staging buffers and a pinned copy of the root stats.
struct ServerLane {
    dvc_ctx* ctx = nullptr;
    int mode = DVC_MODE_ROLLOUT;
    int ctx_index = 0;
    dvc_forest* f = nullptr;
    std::vector<ServerSlot> slots;
    cudaStream_t st = nullptr;
    int32_t* d_slot = nullptr;
    dvc_state* d_root = nullptr;
    int32_t* d_budget = nullptr;
    uint32_t* d_tid = nullptr;
    int32_t* d_stats = nullptr;
    int32_t* h_stats = nullptr;
    int32_t* h_stage = nullptr;  // pinned admission staging: slots, budgets, tree ids, roots
    int resident = 0;
    cudaEvent_t begin = nullptr;  // recorded before a step's search
    cudaEvent_t done = nullptr;   // recorded after the step's statistics reach h_stats
    bool in_flight = false;       // a step of this lane is enqueued and not yet collected
    long long steps = 0;          // steps collected
    double step_us = 0.0;         // their device time (begin to done)
};

// Device bytes of one search slot of context c sized for max_budget
// iterations: node arena (36 B per slot: node, UCB terms, link, creation
// stamp), counting table, plan, meta and pipeline buffers (determinizations
// sampled ahead included), plus the lane's staging per slot.
size_t server_slot_bytes(const dvc_ctx* c, int max_budget) {
    const size_t arena = (size_t)(1 + kRootReserve + 4LL * max_budget) * 36;
    const size_t table = (size_t)(c->cfg.nplayers == 2 ? kDetMaxCells2p : kDetMaxCells) * 8;
    return arena + table + sizeof(DetPlan) + sizeof(TreeMeta) + sizeof(Descent) +
           (sizeof(dvc_state) + sizeof(uint4)) * kDetAhead + 256;
}

}  // namespace

struct dvc_server {
    dvc_ctx* ctx;  // the first context: error messages
    int max_budget;
    std::vector<ServerLane> lanes;
    std::deque<ServerQuery> queue;
    long long completed = 0;
};

namespace {

void lane_free(ServerLane& L) {
    if (L.st) cudaStreamSynchronize(L.st);
    dvc_forest_destroy(L.f);
    L.f = nullptr;
    void* ptrs[] = {L.d_slot, L.d_budget, L.d_tid, L.d_root, L.d_stats};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (L.h_stats) cudaFreeHost(L.h_stats);
    if (L.h_stage) cudaFreeHost(L.h_stage);
    if (L.done) cudaEventDestroy(L.done);
    if (L.begin) cudaEventDestroy(L.begin);
    if (L.st) cudaStreamDestroy(L.st);
    L = ServerLane();
}

// A lane of n slots: staging buffers, idle roots, the forest (budget 0 until
// a query is admitted), and the engine shape for resident searches.
int lane_create(ServerLane& L, dvc_ctx* c, int ctx_index, int mode, int n, int max_budget, uint64_t seed) {
    L.ctx = c;
    L.mode = mode;
    L.ctx_index = ctx_index;
    if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&L.done) != cudaSuccess || cudaEventCreate(&L.begin) != cudaSuccess ||
        cudaMalloc(&L.d_slot, 4 * (size_t)n) != cudaSuccess || cudaMalloc(&L.d_budget, 4 * (size_t)n) != cudaSuccess ||
        cudaMalloc(&L.d_tid, 4 * (size_t)n) != cudaSuccess ||
        cudaMalloc(&L.d_root, sizeof(dvc_state) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&L.d_stats, 32 * (size_t)n) != cudaSuccess ||
        cudaMallocHost(&L.h_stats, 32 * (size_t)n) != cudaSuccess ||
        cudaMallocHost(&L.h_stage, (12 + sizeof(dvc_state)) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DVC_E_OOM, "dvc_server_create: staging buffers");
    }
    // any valid roots: the slots start idle (budget 0) and take real roots on admission
    int rc = dvc_init_states(c, seed, n, L.d_root, L.st);
    if (rc == DVC_OK) {
        std::vector<int32_t> budgets(n, max_budget);
        rc = dvc_forest_create(c, n, L.d_root, budgets.data(), nullptr, seed, &L.f, L.st);
    }
    if (rc == DVC_OK) {
        forest_set_budget_kernel<<<(n + 127) / 128, 128, 0, L.st>>>(L.f->meta, n, 0);
        rc = check_launch(c, "forest_set_budget_kernel");
    }
    // resident searches start and end at any time: the fused engine, one
    // launch per poll over the CTAs that hold resident slots only; four
    // slots per CTA, so a search waits on three others per iteration
    if (rc == DVC_OK && mode == DVC_MODE_ROLLOUT) rc = dvc_forest_tune(L.f, 1, 4, 4, 0);
    if (rc == DVC_OK) L.slots.assign(n, ServerSlot());
    return rc;
}

// Move queued queries of this lane into its free slots (FIFO within the
// lane; a full lane does not hold up the others) and plan their views on
// the device.  Enqueued on the lane's stream; the staging buffers are free
// again once the poll has synchronised that stream.
int lane_admit(dvc_server* sv, int li) {
    ServerLane& L = sv->lanes[li];
    std::vector<int32_t> slot, budget;
    std::vector<dvc_state> root;
    std::vector<uint32_t> tid;
    std::vector<int> freeidx;
    for (int s = 0; s < L.f->n; ++s)
        if (!L.slots[s].busy) freeidx.push_back(s);
    size_t next = 0;
    for (auto it = sv->queue.begin(); it != sv->queue.end() && next < freeidx.size();) {
        if (it->lane != li) {
            ++it;
            continue;
        }
        const int s = freeidx[next++];
        L.slots[s].busy = true;
        L.slots[s].q = *it;
        slot.push_back(s);
        budget.push_back(it->budget);
        root.push_back(it->root);
        tid.push_back((uint32_t)it->id);
        it = sv->queue.erase(it);
    }
    const int k = (int)slot.size();
    L.resident += k;
    if (k == 0) return DVC_OK;
    dvc_ctx* c = L.ctx;
    // pinned staging (the lane is idle: its previous step and copies are done)
    const size_t n = L.slots.size();
    int32_t* hs = L.h_stage;
    int32_t* hb = hs + n;
    uint32_t* ht = (uint32_t*)(hb + n);
    dvc_state* hr = (dvc_state*)(ht + n);
    std::memcpy(hs, slot.data(), 4 * (size_t)k);
    std::memcpy(hb, budget.data(), 4 * (size_t)k);
    std::memcpy(ht, tid.data(), 4 * (size_t)k);
    std::memcpy(hr, root.data(), sizeof(dvc_state) * (size_t)k);
    cudaError_t e = cudaMemcpyAsync(L.d_slot, hs, 4 * k, cudaMemcpyHostToDevice, L.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_budget, hb, 4 * k, cudaMemcpyHostToDevice, L.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_tid, ht, 4 * k, cudaMemcpyHostToDevice, L.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_root, hr, sizeof(dvc_state) * k, cudaMemcpyHostToDevice, L.st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dvc_server admit");
    forest_admit_kernel<<<(k * 32 + 127) / 128, 128, 0, L.st>>>(dev_of(L.f), k, L.d_slot, L.d_root, L.d_budget,
                                                                L.d_tid, L.f->plans, L.f->tables, L.f->table_cap,
                                                                c->cfg.nplayers, c->cfg.ntiles, L.f->pipe.np);
    return check_launch(c, "forest_admit_kernel");
}

}  // namespace

extern "C" {

int dvc_server_create_multi(dvc_ctx* const* ctxs, int n_ctx, const int32_t* h_weights, size_t hbm_budget,
                            int max_budget, int value_share_pct, uint64_t seed, dvc_server** out) {
    if (!ctxs || n_ctx < 1 || n_ctx > 16 || !ctxs[0]) return DVC_E_INVALID;
    dvc_ctx* c0 = ctxs[0];
    if (!out || max_budget < 1 || max_budget > (1 << 24) || value_share_pct < 0 || value_share_pct > 100)
        return fail(c0, DVC_E_INVALID, "dvc_server_create: max_budget 1..2^24, value_share_pct 0..100");
    *out = nullptr;
    long long wsum = 0;
    for (int i = 0; i < n_ctx; ++i) {
        dvc_ctx* c = ctxs[i];
        if (!c) return fail(c0, DVC_E_INVALID, "dvc_server_create: null context");
        if (c->device != c0->device) return fail(c0, DVC_E_INVALID, "dvc_server_create: contexts on different devices");
        if (c->cfg.vanilla)
            return fail(c0, DVC_E_UNSUPPORTED, "dvc_server_create: vanilla trees are searched by forests only");
        for (int j = 0; j < i; ++j)
            if (ctxs[j]->cfg.nplayers == c->cfg.nplayers && ctxs[j]->cfg.ntiles == c->cfg.ntiles)
                return fail(c0, DVC_E_INVALID, "dvc_server_create: two contexts of one game variant");
        const long long w = h_weights ? h_weights[i] : 1;
        if (w < 0) return fail(c0, DVC_E_INVALID, "dvc_server_create: negative weight");
        wsum += w;
    }
    if (wsum <= 0) return fail(c0, DVC_E_INVALID, "dvc_server_create: weights sum to zero");
    if (int rc = set_device(c0)) return rc;
    // slots per (context, mode): the context's share of the HBM budget over
    // its per-slot footprint, value_share_pct of it for value mode
    std::vector<long long> counts(2 * n_ctx, 0);
    long long total_slots = 0;
    for (int i = 0; i < n_ctx; ++i) {
        const long long w = h_weights ? h_weights[i] : 1;
        const double share = (double)hbm_budget * (double)w / (double)wsum;
        const long long n = (long long)(share / (double)server_slot_bytes(ctxs[i], max_budget));
        const long long nv = ctxs[i]->vnet ? n * value_share_pct / 100 : 0;
        counts[2 * i] = n - nv;
        counts[2 * i + 1] = nv;
        if (n - nv > (1 << 20) || nv > (1 << 20))
            return fail(c0, DVC_E_UNSUPPORTED, "dvc_server_create: over 2^20 slots per lane");
        total_slots += n;
    }
    if (total_slots < 1) return fail(c0, DVC_E_OOM, "dvc_server_create: HBM budget below one search slot");
    dvc_server* sv = new (std::nothrow) dvc_server();
    if (!sv) return fail(c0, DVC_E_OOM, "dvc_server_create: host allocation");
    sv->ctx = c0;
    sv->max_budget = max_budget;
    int rc = DVC_OK;
    for (int i = 0; i < n_ctx && rc == DVC_OK; ++i)
        for (int m = 0; m < 2 && rc == DVC_OK; ++m) {
            const int n = (int)counts[2 * i + m];
            if (n < 1) continue;
            sv->lanes.emplace_back();
            rc = lane_create(sv->lanes.back(), ctxs[i], i, m, n, max_budget, seed);
        }
    for (ServerLane& L : sv->lanes)
        if (rc == DVC_OK && L.st && cudaStreamSynchronize(L.st) != cudaSuccess)
            rc = fail(c0, DVC_E_CUDA, "dvc_server_create sync");
    if (rc != DVC_OK) {
        dvc_server_destroy(sv);
        return rc;
    }
    *out = sv;
    return DVC_OK;
}

int dvc_server_create(dvc_ctx* c, size_t hbm_budget, int max_budget, int value_share_pct, uint64_t seed,
                      dvc_server** out) {
    if (!c) return DVC_E_INVALID;
    return dvc_server_create_multi(&c, 1, nullptr, hbm_budget, max_budget, value_share_pct, seed, out);
}

void dvc_server_destroy(dvc_server* sv) {
    if (!sv) return;
    cudaSetDevice(sv->ctx->device);
    for (ServerLane& L : sv->lanes) lane_free(L);
    delete sv;
}

int dvc_server_submit(dvc_server* sv, const dvc_state* h_root, int budget, int mode, uint64_t query_id) {
    if (!sv) return DVC_E_INVALID;
    dvc_ctx* c = sv->ctx;
    if (!h_root || budget < 1 || budget > sv->max_budget || (mode != DVC_MODE_ROLLOUT && mode != DVC_MODE_VALUE))
        return fail(c, DVC_E_INVALID, "dvc_server_submit: root, budget 1..max_budget, mode");
    int lane = -1;
    bool variant = false;
    for (int i = 0; i < (int)sv->lanes.size(); ++i) {
        const ServerLane& L = sv->lanes[i];
        if (L.ctx->cfg.nplayers != h_root->nplayers || L.ctx->cfg.ntiles != h_root->ntiles) continue;
        variant = true;
        if (L.mode == mode) lane = i;
    }
    if (!variant) return fail(c, DVC_E_INVALID, "dvc_server_submit: no context of this root's game variant");
    if (lane < 0) return fail(c, DVC_E_UNSUPPORTED, "dvc_server_submit: no slots for this mode and variant");
    ServerQuery q;
    q.root = *h_root;
    q.budget = budget;
    q.lane = lane;
    q.id = query_id;
    q.t_submit = now_s();
    sv->queue.push_back(q);
    return DVC_OK;
}

int dvc_server_poll(dvc_server* sv, int iterations, dvc_result* h_results, int max_results) {
    if (!sv) return DVC_E_INVALID;
    dvc_ctx* c = sv->ctx;
    if (iterations < 0 || max_results < 0 || (max_results > 0 && !h_results))
        return fail(c, DVC_E_INVALID, "dvc_server_poll: iterations >= 0, results buffer");
    if (int rc = set_device(c)) return rc;
    int written = 0;
    // collect the finished queries of a lane whose step is complete; the lane
    // stays collected-pending while some finished query did not fit
    auto collect = [&](ServerLane& L) -> bool {
        const double t = now_s();
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, L.begin, L.done) == cudaSuccess) {
            L.steps++;
            L.step_us += 1e3 * (double)ms;
        } else {
            cudaGetLastError();
        }
        bool all = true;
        for (int s = 0; s < L.f->n; ++s) {
            ServerSlot& sl = L.slots[s];
            const int32_t* st = L.h_stats + 8 * s;
            if (!sl.busy || st[6] < sl.q.budget) continue;
            if (written >= max_results) {
                all = false;
                break;
            }
            dvc_result& r = h_results[written++];
            r.query_id = sl.q.id;
            r.best_action = st[0];
            r.best_visits = st[1];
            r.best_wins = st[2];
            r.root_visits = st[3];
            r.iterations = st[6];
            r.mode = L.mode;
            r.t_submit = sl.q.t_submit;
            r.t_done = t;
            sl.busy = false;
            L.resident--;
            sv->completed++;
        }
        return all;
    };
    // enqueue admission, `iterations` more of the lane's resident searches
    // and its root statistics on the lane's stream
    auto launch = [&](int li) -> int {
        ServerLane& L = sv->lanes[li];
        if (int rc = lane_admit(sv, li)) return rc;
        if (L.resident == 0) return DVC_OK;
        int top = -1;
        for (int s = 0; s < L.f->n; ++s)
            if (L.slots[s].busy) top = s;
        L.f->active_prefix = top + 1;
        cudaError_t e = cudaEventRecord(L.begin, L.st);
        if (e != cudaSuccess) return cuda_fail(c, e, "dvc_server_poll launch");
        if (iterations > 0)
            if (int rc = dvc_mcts_step(L.f, iterations, L.mode, L.st)) return rc;
        if (int rc = dvc_root_stats(L.f, L.d_stats, L.st)) return rc;
        e = cudaMemcpyAsync(L.h_stats, L.d_stats, 32 * (size_t)L.f->n, cudaMemcpyDeviceToHost, L.st);
        if (e == cudaSuccess) e = cudaEventRecord(L.done, L.st);
        if (e != cudaSuccess) return cuda_fail(c, e, "dvc_server_poll launch");
        L.in_flight = true;
        return DVC_OK;
    };
    // 1. lanes whose step is complete: collect, then relaunch with newly
    //    admitted queries; lanes never stepped or idle: launch
    bool any_done = false;
    for (int li = 0; li < (int)sv->lanes.size(); ++li) {
        ServerLane& L = sv->lanes[li];
        if (L.in_flight) {
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return cuda_fail(c, q, "dvc_server_poll");
            any_done = true;
            if (!collect(L)) continue;  // results left over: collect them next poll first
            L.in_flight = false;
        }
        if (int rc = launch(li)) return rc;
    }
    // 2. if nothing completed yet, wait (host-side) until some lane's step
    //    does, collect it and relaunch it
    bool waiting = !any_done;
    while (waiting) {
        bool flying = false;
        for (int li = 0; li < (int)sv->lanes.size() && waiting; ++li) {
            ServerLane& L = sv->lanes[li];
            if (!L.in_flight) continue;
            flying = true;
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return cuda_fail(c, q, "dvc_server_poll");
            waiting = false;
            if (!collect(L)) break;
            L.in_flight = false;
            if (int rc = launch(li)) return rc;
        }
        if (!flying) break;
        if (waiting) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    return written;
}

int dvc_server_stats(dvc_server* sv, int64_t* h_out) {
    if (!sv || !h_out) return DVC_E_INVALID;
    long long active = 0, rollout = 0, value = 0;
    for (const ServerLane& L : sv->lanes) {
        (L.mode == DVC_MODE_VALUE ? value : rollout) += (long long)L.slots.size();
        active += L.resident;
    }
    h_out[0] = (int64_t)sv->queue.size();
    h_out[1] = active;
    h_out[2] = sv->completed;
    h_out[3] = rollout;
    h_out[4] = value;
    return DVC_OK;
}

int dvc_server_lanes(dvc_server* sv, int max_lanes, int32_t* h_out) {
    if (!sv || max_lanes < 0 || (max_lanes > 0 && !h_out)) return DVC_E_INVALID;
    const int n = (int)sv->lanes.size();
    for (int i = 0; i < n && i < max_lanes; ++i) {
        const ServerLane& L = sv->lanes[i];
        int32_t* o = h_out + 8 * i;
        o[0] = L.ctx_index;
        o[1] = L.ctx->cfg.nplayers;
        o[2] = L.ctx->cfg.ntiles;
        o[3] = L.mode;
        o[4] = (int32_t)L.slots.size();
        o[5] = L.resident;
        o[6] = (int32_t)std::min<long long>(L.steps, INT32_MAX);
        o[7] = (int32_t)std::min<double>(L.step_us / std::max<long long>(L.steps, 1), (double)INT32_MAX);
    }
    return n;
}

}  // extern "C"
