// dvc_tree.cuh -- device-resident UCT trees and one search iteration
// (Sec. II-B: select, expand, simulate, backpropagate; Sec. III-A: node =
// guess (slot, identity), determinized root per simulation, no extra guess in
// the tree, expansion depth limit).
//
// Arena layout, per tree: a slice of 16-byte node slots.  Slot 0 is the root.
// The children of a node live in blocks of consecutive slots -- the root's
// first block is sized to its legal-guess count (fixed for the whole search),
// other nodes' blocks grow 4, 8, 16, 32, 32, ... -- so a warp reads a block
// with one coalesced load.  A block's successor is recorded in `link` at the
// block's first slot.  With blocks no larger than four times the children
// they hold, root block + 4 * budget slots always suffice.
//
// Vanilla MCTS-dvc (Sec. III-A): the root's children are plausible-number
// sets, one per distinct assignment of the tiles the observer cannot see, and
// the guess tree of each hangs below it.  The root's single child block then
// holds `budget` slots (at most one set per iteration), and a per-tree open-
// addressing table maps an assignment to its set node.
#pragma once
#include "dvc_det.cuh"

namespace dvc {

struct Node {
    int32_t visits;
    int32_t wins;
    int32_t child;  // slot of the first child block, -1 if none
    uint32_t meta;  // action code (bits 0-11) | number of children (bits 12-23)
};

struct TreeMeta {
    long long node_off;   // first slot of this tree in the arena
    long long table_off;  // first cell of its determinization table
    int32_t cap;          // slots
    int32_t budget;       // iterations allowed in total
    int32_t done;         // iterations done
    int32_t next_free;    // next unused slot
    int32_t root_legal;   // legal guesses at the root
    uint32_t tree_id;     // stream key
    int32_t failed;       // arena exhausted, or view too large to determinize
    int32_t used;         // nodes in the tree
    long long set_off;    // vanilla: first cell of its plausible-set table
    int32_t set_cells;    // vanilla: cells of that table (2 * budget); 0 otherwise
    int32_t pad_;
};

// A tree's plausible-set table: open addressing with linear probing, cell i
// holds an assignment's key and the slot of its set node (-1: empty).  At
// most `budget` keys in 2 * budget cells, so an empty cell always ends a probe.
struct SetTable {
    uint4* key;
    int32_t* slot;
    uint32_t cells;  // 0: not a vanilla tree
};

// Key of a determinization's plausible-number set as seen by seat obs: the
// other seats' hands in seat order (three words, unused seats zero), then the
// joker gaps and the white-first flag, which place the jokers in the rows.
__device__ __forceinline__ uint4 set_key(const G& g, uint32_t obs) {
    uint32_t h[3] = {0u, 0u, 0u};
    uint32_t k = 0;
#pragma unroll
    for (uint32_t p = 0; p < 4; ++p)
        if (p < g.np && p != obs) h[k++] = g.hand(p);
    return make_uint4(h[0], h[1], h[2], g.jg0 | (g.jg1 << 8) | ((g.jflag & 1u) << 16));
}

// First probe cell of a key: a 64-bit mix (xor-shift-multiply rounds) of its
// words, scaled to the cell count by a multiply-high.
__device__ __forceinline__ uint32_t set_home(const uint4& k, uint32_t cells) {
    unsigned long long a = ((unsigned long long)k.y << 32 | k.x) ^ (((unsigned long long)k.w << 32 | k.z) * 0x9E3779B97F4A7C15ull);
    a ^= a >> 31;
    a *= 0xD6E8FEB86659FD93ull;
    a ^= a >> 32;
    return (uint32_t)(((unsigned long long)(uint32_t)a * cells) >> 32);
}

// Warp-parallel probe: lane j looks at the j-th cell of each round of 32; the
// first cell in probe order that is empty or holds the key ends the probe.
// Returns the set node's slot (-1 if absent) and the cell it sits in, or
// would be inserted into.  Lane-uniform.
__device__ __forceinline__ int32_t set_find(const SetTable& st, const uint4& k, uint32_t& cell) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t home = set_home(k, st.cells);
    for (uint32_t r = 0; r < st.cells; r += 32u) {
        uint32_t c = home + r + lane;
        c = c % st.cells;
        const int32_t s = st.slot[c];
        bool stop = s < 0;
        if (!stop) {
            const uint4 q = st.key[c];
            stop = q.x == k.x && q.y == k.y && q.z == k.z && q.w == k.w;
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, stop);
        if (bal) {
            const uint32_t L = __ffs(bal) - 1u;
            cell = __shfl_sync(0xFFFFFFFFu, c, L);
            return __shfl_sync(0xFFFFFFFFu, s, L);
        }
    }
    cell = 0xFFFFFFFFu;  // unreachable while keys <= cells / 2
    return -1;
}

// Slots reserved for the root's child block: its legal-guess count is
// (face-down slots of opponents) x (unknown identities) <= 25 * 25.
constexpr int32_t kRootReserve = 640;

struct SearchParams {
    uint64_t seed;
    float c_uct;  // UCB1 exploration constant, rounded to float
    int32_t d_max;
    int32_t playouts;
    uint32_t cont_thr;
    int32_t policy;         // playout guesses: 0 uniform, 1 ordering-aware
    int32_t tree_continue;  // 1: a correct in-tree guess keeps the turn (Fig. 2a)
};

__device__ __forceinline__ uint32_t block_size(uint32_t k, bool is_root, uint32_t root_legal) {
    if (is_root && k == 0) return root_legal > 0u ? root_legal : 1u;
    return k >= 3 ? 32u : (4u << k);
}

// What a descent produced: either a node to expand (found = 1, action act)
// or a leaf to score (found = 0).
struct Descent {
    G s;              // state at the node reached
    Rng tr;           // tree stream after the in-tree draws so far
    int32_t node;     // slot reached
    int32_t found;    // 1: expand `act` below `node`
    uint32_t act;
    int32_t nchild;   // children of `node`
    int32_t last_blk, last_size, last_cnt, nblocks;
    int32_t np;       // path length
    uint32_t set_cell;  // vanilla, act == kSet: the table cell for the new set
    uint4 set_key;      // vanilla, act == kSet: its key
};

// Warp-cooperative descent from the root for iteration `it`.  All 32 lanes
// of the calling warp enter with the same arguments and leave with the same
// Descent; lane 0 records the path in path[] / mover[] (shared or global).
// E is a 4 x 26 word scratch (shared memory) for expanded-identity masks.
// ucb[slot] = (wins/n, 1/sqrt(n)) and csl[slot] = c * sqrt(ln n) are the
// node's UCB1 terms, refreshed whenever its counts change (backprop), so a
// selection scan costs one multiply-add per child.  They are the same IEEE
// values a scan would compute from the counts.
// tree0 (optional): the first block of the iteration's tree stream, computed
// ahead of time (the same four words the stream would generate).
// st: the plausible-set table of a vanilla tree.  The determinization's set
// node is the first step below the root; a set not seen before is this
// iteration's expansion (act = kSet) and its leaf is the determinized root.
__device__ __forceinline__ void descend(const G& det, uint32_t obs, const Node* nodes, const int32_t* link,
                                        const float2* ucb, const float* csl_of, const TreeMeta& tm,
                                        const SearchParams& sp, uint32_t it, int32_t* path, uint8_t* mover,
                                        uint32_t* E, Descent& d, const uint4* tree0 = nullptr,
                                        const SetTable& st = SetTable{nullptr, nullptr, 0u}) {
    const uint32_t lane = threadIdx.x & 31u;
    d.s = det;
    d.tr.open(sp.seed, tm.tree_id, 0u, it, kTagTree);
    if (tree0) d.tr.preload(*tree0);
    d.node = 0;
    d.found = 0;
    d.np = 1;
    if (lane == 0) {
        path[0] = 0;
        mover[0] = (uint8_t)obs;
    }
    uint32_t depth = 0;
    if (st.cells) {
        const uint4 key = set_key(d.s, obs);
        uint32_t cell;
        const int32_t slot = set_find(st, key, cell);
        if (slot < 0) {
            // a new set: appended to the root's single child block
            const Node r = nodes[0];
            const int32_t nsets = (int32_t)(r.meta >> 12);
            d.found = 1;
            d.act = kSet;
            d.set_cell = cell;
            d.set_key = key;
            d.nchild = nsets;
            d.nblocks = nsets ? 1 : 0;
            d.last_blk = nsets ? r.child : -1;
            d.last_size = tm.root_legal;
            d.last_cnt = nsets;
            return;
        }
        if (lane == 0) {
            path[1] = slot;
            mover[1] = (uint8_t)obs;
        }
        d.np = 2;
        d.node = slot;
    }
    while (d.s.winner == kNone && depth < (uint32_t)sp.d_max) {
        // loads that do not depend on one another are issued together: the
        // node and its exploration term; below, each child with its UCB1
        // terms, and the next block's start before this block is scanned
        const Node nd = nodes[d.node];
        const float csl_node = csl_of[d.node];  // any slot's entry exists; used only if it has children
        const uint32_t nchild = nd.meta >> 12;
        const uint32_t cur = d.s.cur;
        const uint32_t U = d.s.tmask & ~d.s.hand(cur) & ~d.s.rev;
        for (uint32_t e = lane; e < 104u; e += 32u) E[e] = 0u;
        __syncwarp();
        const float csl = nchild ? csl_node : 0.0f;
        float best_sc = -1.0f;
        uint32_t best_rank = 0xFFFFFFFFu;
        int32_t best_slot = -1;
        uint32_t best_code = 0;
        int32_t blk = nd.child;
        uint32_t seen = 0, k = 0;
        bool stop_child = false;  // this lane saw the node's STOP child
        d.last_blk = -1;
        d.last_size = 0;
        d.last_cnt = 0;
        while (seen < nchild) {
            const uint32_t size = block_size(k, d.node == 0, (uint32_t)tm.root_legal);
            const uint32_t cnt = min(size, nchild - seen);
            const int32_t next_blk = seen + cnt < nchild ? link[blk] : -1;
            for (uint32_t e = lane; e < cnt; e += 32u) {
                const Node ch = nodes[blk + (int32_t)e];
                const float2 u = ucb[blk + (int32_t)e];  // set by the child's first backprop
                const uint32_t code = ch.meta & 0xFFFu;
                const uint32_t q = code >> 10, sl = (code >> 5) & 31u, x = code & 31u;
                stop_child |= code == kStop;
                if (code != kStop && sl < 26u) atomicOr(&E[q * 26u + sl], 1u << x);
                if (action_legal(d.s, code)) {
                    const float sc = __fadd_rn(u.x, __fmul_rn(csl, u.y));
                    const uint32_t rk = canon_rank(code, cur, d.s.np);
                    if (best_slot < 0 || sc > best_sc || (sc == best_sc && rk < best_rank)) {
                        best_sc = sc;
                        best_rank = rk;
                        best_slot = blk + (int32_t)e;
                        best_code = code;
                    }
                }
            }
            seen += cnt;
            d.last_blk = blk;
            d.last_size = (int32_t)size;
            d.last_cnt = (int32_t)cnt;
            ++k;
            if (seen < nchild) blk = next_blk;
        }
        d.nblocks = (int32_t)k;
        d.nchild = (int32_t)nchild;
        __syncwarp();
        // first legal action without a child, canonical order (STOP first)
        uint32_t act = 0;
        bool found = false;
        if (d.s.mstop && !__any_sync(0xFFFFFFFFu, stop_child)) {
            act = kStop;
            found = true;
        }
        for (uint32_t off = 1; off < d.s.np && !found; ++off) {
            uint32_t q = cur + off;
            q = q >= d.s.np ? q - d.s.np : q;
            if (!((d.s.alive >> q) & 1u)) continue;
            const uint32_t nh = __popc(d.s.hand(q) & ~d.s.rev);
            for (uint32_t h0 = 0; h0 < nh && !found; h0 += 32u) {
                const uint32_t h = h0 + lane;
                uint32_t avail = 0u, sp_ = 0u;
                if (h < nh) {
                    const uint32_t t = hidden_slot(d.s, q, h);
                    sp_ = seq_pos(d.s, q, t);
                    if (sp_ < 26u) avail = U & ~E[q * 26u + sp_];
                }
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, avail != 0u);
                if (bal) {
                    const uint32_t L = __ffs(bal) - 1u;
                    const uint32_t spL = __shfl_sync(0xFFFFFFFFu, sp_, L);
                    const uint32_t avL = __shfl_sync(0xFFFFFFFFu, avail, L);
                    act = (q << 10) | (spL << 5) | ((uint32_t)__ffs(avL) - 1u);
                    found = true;
                }
            }
        }
        if (found) {
            d.found = 1;
            d.act = act;
            return;
        }
        // UCB1 argmax over lanes: higher score, then lower canonical rank
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float osc = __shfl_xor_sync(0xFFFFFFFFu, best_sc, o);
            const uint32_t ork = __shfl_xor_sync(0xFFFFFFFFu, best_rank, o);
            const int32_t osl = __shfl_xor_sync(0xFFFFFFFFu, best_slot, o);
            const uint32_t ocd = __shfl_xor_sync(0xFFFFFFFFu, best_code, o);
            const bool take = osl >= 0 && (best_slot < 0 || osc > best_sc || (osc == best_sc && ork < best_rank));
            if (take) {
                best_sc = osc;
                best_rank = ork;
                best_slot = osl;
                best_code = ocd;
            }
        }
        const uint32_t who = d.s.cur;
        tree_apply(d.s, best_code, d.tr, sp.tree_continue != 0);
        if (lane == 0) {
            path[d.np] = best_slot;
            mover[d.np] = (uint8_t)who;
        }
        d.np++;
        d.node = best_slot;
        ++depth;
    }
}

// Create the child found by descend() and step the state through its action
// (a new plausible set is entered in the tree's set table and leaves the state
// as it is).  Lane-uniform; lane 0 writes memory.  next_free is the tree's
// allocator (uniform register copy).  Returns false if the arena is exhausted.
__device__ __forceinline__ bool expand_child(Descent& d, Node* nodes, int32_t* link, int32_t* created,
                                             const TreeMeta& tm, int32_t& next_free, int32_t& used, uint32_t it,
                                             int32_t* path, uint8_t* mover, bool cont,
                                             const SetTable& st = SetTable{nullptr, nullptr, 0u}) {
    const uint32_t lane = threadIdx.x & 31u;
    int32_t slot;
    if (d.nchild == 0 || d.last_cnt >= d.last_size) {
        // a new child block: first block of this node, or the last one is full
        const uint32_t k = d.nchild == 0 ? 0u : (uint32_t)d.nblocks;
        const int32_t size = (int32_t)block_size(k, d.node == 0, (uint32_t)tm.root_legal);
        if (next_free + size > tm.cap) return false;
        slot = next_free;
        next_free += size;
        for (int32_t e = (int32_t)lane; e < size; e += 32) created[slot + e] = -1;  // slots not yet nodes
        if (lane == 0) {
            if (d.nchild == 0) nodes[d.node].child = slot;
            else link[d.last_blk] = slot;
            link[slot] = -1;
        }
    } else {
        slot = d.last_blk + d.last_cnt;
    }
    if (lane == 0) {
        Node c;
        c.visits = 0;
        c.wins = 0;
        c.child = -1;
        c.meta = d.act;
        nodes[slot] = c;
        created[slot] = (int32_t)it;
        nodes[d.node].meta += 1u << 12;
        path[d.np] = slot;
        mover[d.np] = (uint8_t)d.s.cur;
        if (d.act == kSet) {
            st.key[d.set_cell] = d.set_key;
            st.slot[d.set_cell] = slot;
        }
    }
    if (d.act != kSet) tree_apply(d.s, d.act, d.tr, cont);
    d.np++;
    d.node = slot;
    ++used;
    return true;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Backpropagation (Sec. II-B): every node on the path gains `playouts` visits
// and the playouts won by the seat that moved into it.
__device__ __forceinline__ void backprop(Node* nodes, float2* ucb, float* csl, const int32_t* path,
                                         const uint8_t* mover, int32_t np, const int32_t* wins, int32_t playouts,
                                         float c_uct) {
    const uint32_t lane = threadIdx.x & 31u;
    for (int32_t e = (int32_t)lane; e < np; e += 32) {
        const int32_t slot = path[e];
        Node* n = &nodes[slot];
        const int32_t v = n->visits + playouts;
        const int32_t w = n->wins + wins[mover[e]];
        n->visits = v;
        n->wins = w;
        const float dv = __int2float_rn(v);
        ucb[slot] = make_float2(__fdiv_rn(__int2float_rn(w), dv), __fdiv_rn(1.0f, __fsqrt_rn(dv)));
        csl[slot] = __fmul_rn(c_uct, __fsqrt_rn(ln_series(dv)));
    }
}

}  // namespace dvc
