// dvc_det.cuh -- uniform determinization of a root view (Sec. III-A: the
// plausible values of the tiles a player cannot see are re-drawn for every
// simulation), on the device.
//
// The unknown tiles (not in the observer's hand, not face up) are spread
// over the opponents' face-down slots and the pool.  A consistent deal keeps
// each opponent's face-up tiles where they are and its numbered tiles in
// ascending order; jokers may stand in any slot.  For opponent k the face-down
// slots between consecutive face-up numbered tiles ("anchors") form gaps; a
// gap takes numbered tiles from its id interval in order, and slots a gap
// still has open when the ascending walk over unknown numbered tiles passes
// its right anchor must hold jokers.  F(i, r, J) counts completions when the
// unknown numbered tile u_i is next, gap slots r[k] are still open and J
// unknown jokers are unplaced; closing a gap of c slots with o open ones
// multiplies by C(c, o) * J!/(J-o)!.  The table depends only on the root
// view, so it is filled once per search and sampled every iteration: walk
// the tiles in id order, pick the destination (pool first, then opponents from
// observer+1) with weight = completions it leaves, as floor(r64 * W / 2^64)
// from two stream words, and pick each close's joker slots the same way.
#pragma once
#include "dvc_device.cuh"

namespace dvc {

constexpr uint32_t kDetMaxCells = 32768;  // table capacity for 3-4 players
constexpr uint32_t kDetMaxCells2p = 2048;  // two players: (m+1)(gap+1)(J+1) <= 25*25*3

struct DetPlan {
    uint8_t nq, m, J0, obs;
    uint8_t q[3];
    uint8_t nanch[3];
    uint8_t u[24];
    uint8_t jok[2];
    uint8_t gapsz[3][25];
    uint8_t G[3][25];
    uint8_t seqlen[3];
    uint8_t tpl[3][26];  // face-up slot: tile id; face-down slot: 0x80 | gap
    uint8_t pad[2];
    uint32_t off[26];    // first cell of layer i (i = 0..m), off[m+1] = cells
    uint32_t cells;
    uint32_t ok;         // 1 if the table fits
    unsigned long long total;
};

// Left-to-right tiles of hand p.
__device__ __forceinline__ uint32_t hand_sequence(const G& g, uint32_t p, uint8_t* out) {
    const uint32_t hp = g.hand(p);
    const uint32_t n = __popc(hp);
    for (uint32_t s = 0; s < n; ++s) out[s] = (uint8_t)seq_tile(g, p, s);
    return n;
}

__device__ __forceinline__ uint32_t det_rad(const DetPlan& pl, uint32_t k, uint32_t i) {
    return k < pl.nq ? (uint32_t)pl.gapsz[k][pl.G[k][i]] + 1u : 1u;
}

__device__ __forceinline__ uint32_t det_cell(const DetPlan& pl, uint32_t i, const uint32_t* r, uint32_t J) {
    const uint32_t r0 = det_rad(pl, 0, i), r1 = det_rad(pl, 1, i), r2 = det_rad(pl, 2, i);
    return pl.off[i] + ((J * r0 + r[0]) * r1 + r[1]) * r2 + r[2];
}

// Ways to put o jokers into a gap of c slots, choosing from J distinct jokers.
__device__ __forceinline__ unsigned long long joker_ways(uint32_t c, uint32_t o, uint32_t J) {
    if (o == 0) return 1ull;
    if (o > J || o > c) return 0ull;
    if (o == 1) return (unsigned long long)c * J;
    return (unsigned long long)(c * (c - 1u) / 2u) * 2ull;  // o == 2, J == 2
}

// Pass from layer i to i+1 (i = -1: from the start to layer 0).  Returns the
// product of the close factors (0: no completion) and updates r, J.
__device__ __forceinline__ unsigned long long det_pass(const DetPlan& pl, int i, uint32_t* r, uint32_t& J) {
    unsigned long long mult = 1ull;
    for (uint32_t k = 0; k < pl.nq; ++k) {
        const int from = i < 0 ? -1 : (int)pl.G[k][i];
        const int to = pl.G[k][i + 1];
        if (to == from) continue;
        for (int gg = from < 0 ? 0 : from; gg < to; ++gg) {
            const uint32_t c = pl.gapsz[k][gg];
            const uint32_t open = gg == from ? r[k] : c;
            const unsigned long long f = joker_ways(c, open, J);
            if (!f) return 0ull;
            J -= open;
            mult *= f;
        }
        r[k] = pl.gapsz[k][to];
    }
    return mult;
}

__device__ __forceinline__ unsigned long long det_finish(const DetPlan& pl, const uint32_t* r, uint32_t J) {
    unsigned long long mult = 1ull;
    for (uint32_t k = 0; k < pl.nq; ++k) {
        const unsigned long long f = joker_ways(pl.gapsz[k][pl.nanch[k]], r[k], J);
        if (!f) return 0ull;
        J -= r[k];
        mult *= f;
    }
    return mult;
}

// Build the plan of the view of `obs` (a seat) in state g.
__device__ __forceinline__ void det_plan(const G& g, uint32_t obs, DetPlan& pl) {
    if (obs >= g.np) obs = g.cur;
    pl.nq = (uint8_t)(g.np - 1u);
    pl.obs = (uint8_t)obs;
    for (uint32_t k = 0; k < 3; ++k) {
        pl.nanch[k] = 0;
        pl.seqlen[k] = 0;
        for (uint32_t a = 0; a < 25; ++a) {
            pl.gapsz[k][a] = 0;
            pl.G[k][a] = 0;
        }
    }
    for (uint32_t k = 0; k < pl.nq; ++k) {
        uint32_t q = obs + 1u + k;
        q = q >= g.np ? q - g.np : q;
        pl.q[k] = (uint8_t)q;
        uint8_t seq[26];
        const uint32_t n = hand_sequence(g, q, seq);
        pl.seqlen[k] = (uint8_t)n;
        uint32_t gap = 0;
        for (uint32_t s = 0; s < n; ++s) {
            const uint32_t t = seq[s];
            if ((g.rev >> t) & 1u) {
                pl.tpl[k][s] = (uint8_t)t;
                if (t < 24u) ++gap;
            } else {
                pl.tpl[k][s] = (uint8_t)(0x80u | gap);
                pl.gapsz[k][gap]++;
            }
        }
        pl.nanch[k] = (uint8_t)gap;
    }
    const uint32_t unk = g.tmask & ~g.hand(obs) & ~g.rev;
    uint32_t m = 0;
    uint32_t rest = unk & kNumMask;
    while (rest) {
        const uint32_t t = __ffs(rest) - 1;
        pl.u[m++] = (uint8_t)t;
        rest &= rest - 1u;
    }
    pl.m = (uint8_t)m;
    pl.J0 = 0;
    if ((unk >> 24) & 1u) pl.jok[pl.J0++] = 24;
    if ((unk >> 25) & 1u) pl.jok[pl.J0++] = 25;
    for (uint32_t k = 0; k < pl.nq; ++k) {
        // anchors of seat k ascending = face-up numbered tiles of its template
        for (uint32_t i = 0; i <= m; ++i) {
            if (i == m) {
                pl.G[k][i] = pl.nanch[k];
                continue;
            }
            uint32_t gcount = 0;
            for (uint32_t s = 0; s < pl.seqlen[k]; ++s) {
                const uint32_t t = pl.tpl[k][s];
                if (!(t & 0x80u) && t < 24u && t < pl.u[i]) ++gcount;
            }
            pl.G[k][i] = (uint8_t)gcount;
        }
    }
    uint32_t off = 0;
    for (uint32_t i = 0; i <= m; ++i) {
        pl.off[i] = off;
        off += (pl.J0 + 1u) * det_rad(pl, 0, i) * det_rad(pl, 1, i) * det_rad(pl, 2, i);
    }
    pl.off[m + 1] = off;
    pl.cells = off;
    pl.ok = off <= kDetMaxCells ? 1u : 0u;
    pl.total = 0ull;
}

// Fill the counting table F (pl.cells entries) for layers m down to 0, cells
// of one layer split over `nthr` cooperating threads (thread `tid`); `sync`
// must be a barrier over those threads.  Sets pl.total (by thread 0).
template <typename Sync>
__device__ void det_fill(DetPlan& pl, unsigned long long* F, uint32_t tid, uint32_t nthr, Sync sync) {
    for (int i = pl.m; i >= 0; --i) {
        const uint32_t r0 = det_rad(pl, 0, i), r1 = det_rad(pl, 1, i), r2 = det_rad(pl, 2, i);
        const uint32_t ncell = (pl.J0 + 1u) * r0 * r1 * r2;
        for (uint32_t c = tid; c < ncell; c += nthr) {
            uint32_t rem = c;
            uint32_t r[3];
            r[2] = rem % r2;
            rem /= r2;
            r[1] = rem % r1;
            rem /= r1;
            r[0] = rem % r0;
            const uint32_t J = rem / r0;
            unsigned long long v = 0ull;
            if (i == pl.m) {
                v = det_finish(pl, r, J);
            } else {
                for (int d = -1; d < (int)pl.nq; ++d) {
                    uint32_t rr[3] = {r[0], r[1], r[2]};
                    uint32_t JJ = J;
                    if (d >= 0) {
                        if (rr[d] == 0) continue;
                        rr[d]--;
                    }
                    const unsigned long long f = det_pass(pl, i, rr, JJ);
                    if (f) v += f * F[det_cell(pl, i + 1, rr, JJ)];
                }
            }
            F[pl.off[i] + c] = v;
        }
        sync();
    }
    if (tid == 0) {
        uint32_t r[3] = {0, 0, 0};
        uint32_t J = pl.J0;
        const unsigned long long f = det_pass(pl, -1, r, J);
        pl.total = f ? f * F[det_cell(pl, 0, r, J)] : 0ull;
    }
    sync();
}

// Joker slots chosen while sampling: per opponent, per gap-local slot.
struct JokerPick {
    uint8_t n;
    uint8_t k[2], gap[2], local[2], id[2];
};

// Choose which open slots of a closing gap hold jokers, and which jokers.
__device__ __forceinline__ void det_place(uint32_t k, uint32_t gap, uint32_t c, uint32_t open, uint32_t& J,
                                          uint32_t* jleft, Rng& rng, JokerPick& jp) {
    const unsigned long long opts = joker_ways(c, open, J);
    if (opts == 0ull || open > 2u || jp.n + open > 2u) return;  // only for a view with no completion
    const unsigned long long z = pick64(rng.next64(), opts);
    const unsigned long long perms = open == 1 ? J : 2ull;
    const unsigned long long posidx = z / perms, perm = z % perms;
    uint32_t pos0 = 0, pos1 = 0;
    if (open == 1) {
        pos0 = (uint32_t)posidx;
    } else {
        unsigned long long left = posidx;
        for (uint32_t a = 0; a < c; ++a) {
            const unsigned long long cnt = c - 1u - a;
            if (left < cnt) {
                pos0 = a;
                pos1 = a + 1u + (uint32_t)left;
                break;
            }
            left -= cnt;
        }
    }
    uint32_t id0, id1 = 0;
    if (open == 1) {
        id0 = jleft[perm];
    } else {
        id0 = jleft[perm == 0 ? 0 : 1];
        id1 = jleft[perm == 0 ? 1 : 0];
    }
    jp.k[jp.n] = (uint8_t)k;
    jp.gap[jp.n] = (uint8_t)gap;
    jp.local[jp.n] = (uint8_t)pos0;
    jp.id[jp.n] = (uint8_t)id0;
    jp.n++;
    if (open == 2) {
        jp.k[jp.n] = (uint8_t)k;
        jp.gap[jp.n] = (uint8_t)gap;
        jp.local[jp.n] = (uint8_t)pos1;
        jp.id[jp.n] = (uint8_t)id1;
        jp.n++;
    }
    // drop the chosen jokers from the ascending list of unplaced ones
    uint32_t keep[2], nk = 0;
    for (uint32_t a = 0; a < J; ++a) {
        const bool used = jleft[a] == id0 || (open == 2 && jleft[a] == id1);
        if (!used) keep[nk++] = jleft[a];
    }
    for (uint32_t a = 0; a < nk; ++a) jleft[a] = keep[a];
    J = nk;
}

// det_pass with joker placement on each close.
__device__ __forceinline__ void det_pass_sample(const DetPlan& pl, int i, uint32_t* r, uint32_t& J, uint32_t* jleft,
                                                Rng& rng, JokerPick& jp) {
    for (uint32_t k = 0; k < pl.nq; ++k) {
        const int from = i < 0 ? -1 : (int)pl.G[k][i];
        const int to = pl.G[k][i + 1];
        if (to == from) continue;
        for (int gg = from < 0 ? 0 : from; gg < to; ++gg) {
            const uint32_t c = pl.gapsz[k][gg];
            const uint32_t open = gg == from ? r[k] : c;
            if (open) det_place(k, gg, c, open, J, jleft, rng, jp);
        }
        r[k] = pl.gapsz[k][to];
    }
}

// Sample one determinization of root g (whose view pl describes) into out.
__device__ __forceinline__ void det_sample(const DetPlan& pl, const unsigned long long* F, const G& g, Rng& rng,
                                           G& out) {
    if (!pl.ok || pl.total == 0ull) {  // no consistent deal: leave the state as it is
        out = g;
        return;
    }
    uint32_t r[3] = {0, 0, 0};
    uint32_t J = pl.J0;
    uint32_t jleft[2] = {pl.jok[0], pl.jok[1]};
    JokerPick jp;
    jp.n = 0;
    uint32_t got[3] = {0, 0, 0};  // numbered tiles dealt to each opponent (bitmask)
    det_pass_sample(pl, -1, r, J, jleft, rng, jp);
    for (uint32_t i = 0; i < pl.m; ++i) {
        unsigned long long w[4] = {0ull, 0ull, 0ull, 0ull}, W = 0ull;
        for (int d = -1; d < (int)pl.nq; ++d) {
            uint32_t rr[3] = {r[0], r[1], r[2]};
            uint32_t JJ = J;
            if (d >= 0) {
                if (rr[d] == 0) continue;
                rr[d]--;
            }
            const unsigned long long f = det_pass(pl, (int)i, rr, JJ);
            const unsigned long long v = f ? f * F[det_cell(pl, i + 1, rr, JJ)] : 0ull;
            w[d + 1] = v;
            W += v;
        }
        unsigned long long x = pick64(rng.next64(), W);
        int dest = -1;
        for (int e = 0; e < 4; ++e) {
            if (x < w[e]) {
                dest = e - 1;
                break;
            }
            x -= w[e];
        }
        if (dest >= 0) {
            got[dest] |= 1u << pl.u[i];
            r[dest]--;
        }
        det_pass_sample(pl, (int)i, r, J, jleft, rng, jp);
    }
    for (uint32_t k = 0; k < pl.nq; ++k) {
        const uint32_t gg = pl.nanch[k];
        if (r[k]) det_place(k, gg, pl.gapsz[k][gg], r[k], J, jleft, rng, jp);
    }
    // Rebuild the opponents' hands from their templates.
    out = g;
    uint32_t jown[2] = {0xFFu, 0xFFu}, jgap[2] = {0u, 0u}, jseq[2] = {0u, 0u};
    for (uint32_t j = 0; j < 2; ++j) {
        const uint32_t bit = 1u << (24u + j);
        if (g.hand(pl.obs) & bit) {
            jown[j] = pl.obs;
            jgap[j] = j ? g.jg1 : g.jg0;
            jseq[j] = joker_pos(g, g.hand(pl.obs), j);
        }
    }
    for (uint32_t k = 0; k < pl.nq; ++k) {
        const uint32_t q = pl.q[k];
        uint32_t hand = 0u, numbered = 0u;
        uint32_t rest = got[k];
        uint32_t local[25];
        for (uint32_t a = 0; a < 25; ++a) local[a] = 0u;
        for (uint32_t s = 0; s < pl.seqlen[k]; ++s) {
            const uint32_t slot = pl.tpl[k][s];
            uint32_t t;
            if (!(slot & 0x80u)) {
                t = slot;
            } else {
                const uint32_t gg = slot & 0x7Fu;
                const uint32_t li = local[gg]++;
                t = 0xFFu;
                for (uint32_t e = 0; e < jp.n; ++e)
                    if (jp.k[e] == k && jp.gap[e] == gg && jp.local[e] == li) t = jp.id[e];
                if (t == 0xFFu) {
                    if (!rest) continue;  // unreachable for a deal drawn with positive weight
                    t = __ffs(rest) - 1u;
                    rest &= rest - 1u;
                }
            }
            hand |= 1u << t;
            if (t >= 24u && t < 26u) {
                jown[t - 24u] = q;
                jgap[t - 24u] = numbered;
                jseq[t - 24u] = s;
            } else {
                ++numbered;
            }
        }
        if (q == 0) out.h0 = hand;
        if (q == 1) out.h1 = hand;
        if (q == 2) out.h2 = hand;
        if (q == 3) out.h3 = hand;
    }
    out.jg0 = jown[0] == 0xFFu ? 0u : jgap[0];
    out.jg1 = jown[1] == 0xFFu ? 0u : jgap[1];
    out.jflag = (jown[0] != 0xFFu && jown[0] == jown[1] && jgap[0] == jgap[1] && jseq[1] < jseq[0]) ? 1u : 0u;
}

}  // namespace dvc
