// dvc_device.cuh -- device-side game core of the Da Vinci Code MCTS engine
// (arXiv 2403.10720): counter-based random streams, the packed game state,
// the rules of Sec. II-A and the random playout of Sec. II-B.
//
// State lives in registers as tile bitmasks.  A hand's left-to-right order is
// derived: numbered tiles by id, each joker after `gap` numbered tiles, two
// jokers with the same gap ordered by one flag bit.  Every random choice is a
// uniform index floor(w * n / 2^32) over a canonical enumeration, taken from
// the next word of the playout's own Philox stream, so results depend only
// on (seed, tree, iteration, playout) and never on thread placement.
#pragma once
#include <stdint.h>

#include "../../include/dvc.h"

namespace dvc {

constexpr uint32_t kNumMask = 0x00FFFFFFu;  // numbered tiles 0..23
constexpr uint32_t kJokerMask = 0x03000000u;
constexpr uint32_t kNone = 0xFFu;
constexpr uint32_t kTagInit = 1, kTagDet = 2, kTagTree = 3, kTagRoll = 4, kTagPlay = 5;
// STOP (Fig. 2a): end a turn after a correct guess.  Guesses are coded
// seat << 10 | slot << 5 | identity.
constexpr uint32_t kStop = 0xFFFu;
constexpr uint32_t kSet = 0xFFEu;  // action code of a plausible-number-set node (vanilla MCTS-dvc)
// Two-player fast path: `winner` holds kPend while a playout that began where
// the mover may stop has still to draw its continue coin.
constexpr uint32_t kPend = 0xFEu;

// ------------------------------------------------------------------ Philox
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the halves crossed and the round key xored in;
// the key advances by the two Weyl constants between rounds.
__device__ __forceinline__ void philox10(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3, uint32_t k0,
                                         uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
        const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
        const uint32_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
        x0 = n0;
        x1 = lo1;
        x2 = n2;
        x3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// A stream: key (seed low word, tree), counter (block, j, i, tag word).  The
// four words of a block are handed out in order through a small shift queue.
struct Rng {
    uint32_t k0, k1, blk, j, i, tw;
    uint32_t w0, w1, w2, w3;
    uint32_t left;   // words left in the queue
    uint32_t count;  // words handed out (work statistics)

    __device__ __forceinline__ void open(uint64_t seed, uint32_t tree, uint32_t jj, uint32_t ii, uint32_t tag) {
        k0 = (uint32_t)seed;
        k1 = tree;
        blk = 0;
        j = jj;
        i = ii;
        tw = tag + 16u * (uint32_t)(seed >> 32);
        left = 0;
        count = 0;
    }
    __device__ __forceinline__ void ensure(uint32_t) {}  // next() refills by itself
    __device__ __forceinline__ void refill() {
        uint32_t a = blk, b = j, c = i, d = tw;
        philox10(a, b, c, d, k0, k1);
        w0 = a;
        w1 = b;
        w2 = c;
        w3 = d;
        left = 4;
        ++blk;
    }
    // Take block 0 as computed elsewhere (e.g. ahead of time); right after open().
    __device__ __forceinline__ void preload(uint4 b0) {
        w0 = b0.x;
        w1 = b0.y;
        w2 = b0.z;
        w3 = b0.w;
        left = 4;
        blk = 1;
    }
    // Block 0 of a stream, as refill() computes it.
    __device__ __forceinline__ uint4 block0() const {
        uint32_t a = 0u, b = j, c = i, d = tw;
        philox10(a, b, c, d, k0, k1);
        return make_uint4(a, b, c, d);
    }
    __device__ __forceinline__ uint32_t next() {
        if (left == 0) refill();
        const uint32_t r = w0;
        w0 = w1;
        w1 = w2;
        w2 = w3;
        --left;
        ++count;
        return r;
    }
    __device__ __forceinline__ uint64_t next64() {
        const uint64_t lo = next();
        const uint64_t hi = next();
        return (hi << 32) | lo;
    }
};

__device__ __forceinline__ uint32_t pick(uint32_t w, uint32_t n) { return __umulhi(w, n); }
__device__ __forceinline__ uint64_t pick64(uint64_t r, uint64_t n) { return __umul64hi(r, n); }

// Position of the r-th set bit (r = 0..7) of each byte value, 4 bits per rank.
__device__ const uint32_t kSelectInByte[256] = {
    0x00000000u, 0x00000000u, 0x00000001u, 0x00000010u, 0x00000002u, 0x00000020u, 0x00000021u, 0x00000210u,
    0x00000003u, 0x00000030u, 0x00000031u, 0x00000310u, 0x00000032u, 0x00000320u, 0x00000321u, 0x00003210u,
    0x00000004u, 0x00000040u, 0x00000041u, 0x00000410u, 0x00000042u, 0x00000420u, 0x00000421u, 0x00004210u,
    0x00000043u, 0x00000430u, 0x00000431u, 0x00004310u, 0x00000432u, 0x00004320u, 0x00004321u, 0x00043210u,
    0x00000005u, 0x00000050u, 0x00000051u, 0x00000510u, 0x00000052u, 0x00000520u, 0x00000521u, 0x00005210u,
    0x00000053u, 0x00000530u, 0x00000531u, 0x00005310u, 0x00000532u, 0x00005320u, 0x00005321u, 0x00053210u,
    0x00000054u, 0x00000540u, 0x00000541u, 0x00005410u, 0x00000542u, 0x00005420u, 0x00005421u, 0x00054210u,
    0x00000543u, 0x00005430u, 0x00005431u, 0x00054310u, 0x00005432u, 0x00054320u, 0x00054321u, 0x00543210u,
    0x00000006u, 0x00000060u, 0x00000061u, 0x00000610u, 0x00000062u, 0x00000620u, 0x00000621u, 0x00006210u,
    0x00000063u, 0x00000630u, 0x00000631u, 0x00006310u, 0x00000632u, 0x00006320u, 0x00006321u, 0x00063210u,
    0x00000064u, 0x00000640u, 0x00000641u, 0x00006410u, 0x00000642u, 0x00006420u, 0x00006421u, 0x00064210u,
    0x00000643u, 0x00006430u, 0x00006431u, 0x00064310u, 0x00006432u, 0x00064320u, 0x00064321u, 0x00643210u,
    0x00000065u, 0x00000650u, 0x00000651u, 0x00006510u, 0x00000652u, 0x00006520u, 0x00006521u, 0x00065210u,
    0x00000653u, 0x00006530u, 0x00006531u, 0x00065310u, 0x00006532u, 0x00065320u, 0x00065321u, 0x00653210u,
    0x00000654u, 0x00006540u, 0x00006541u, 0x00065410u, 0x00006542u, 0x00065420u, 0x00065421u, 0x00654210u,
    0x00006543u, 0x00065430u, 0x00065431u, 0x00654310u, 0x00065432u, 0x00654320u, 0x00654321u, 0x06543210u,
    0x00000007u, 0x00000070u, 0x00000071u, 0x00000710u, 0x00000072u, 0x00000720u, 0x00000721u, 0x00007210u,
    0x00000073u, 0x00000730u, 0x00000731u, 0x00007310u, 0x00000732u, 0x00007320u, 0x00007321u, 0x00073210u,
    0x00000074u, 0x00000740u, 0x00000741u, 0x00007410u, 0x00000742u, 0x00007420u, 0x00007421u, 0x00074210u,
    0x00000743u, 0x00007430u, 0x00007431u, 0x00074310u, 0x00007432u, 0x00074320u, 0x00074321u, 0x00743210u,
    0x00000075u, 0x00000750u, 0x00000751u, 0x00007510u, 0x00000752u, 0x00007520u, 0x00007521u, 0x00075210u,
    0x00000753u, 0x00007530u, 0x00007531u, 0x00075310u, 0x00007532u, 0x00075320u, 0x00075321u, 0x00753210u,
    0x00000754u, 0x00007540u, 0x00007541u, 0x00075410u, 0x00007542u, 0x00075420u, 0x00075421u, 0x00754210u,
    0x00007543u, 0x00075430u, 0x00075431u, 0x00754310u, 0x00075432u, 0x00754320u, 0x00754321u, 0x07543210u,
    0x00000076u, 0x00000760u, 0x00000761u, 0x00007610u, 0x00000762u, 0x00007620u, 0x00007621u, 0x00076210u,
    0x00000763u, 0x00007630u, 0x00007631u, 0x00076310u, 0x00007632u, 0x00076320u, 0x00076321u, 0x00763210u,
    0x00000764u, 0x00007640u, 0x00007641u, 0x00076410u, 0x00007642u, 0x00076420u, 0x00076421u, 0x00764210u,
    0x00007643u, 0x00076430u, 0x00076431u, 0x00764310u, 0x00076432u, 0x00764320u, 0x00764321u, 0x07643210u,
    0x00000765u, 0x00007650u, 0x00007651u, 0x00076510u, 0x00007652u, 0x00076520u, 0x00076521u, 0x00765210u,
    0x00007653u, 0x00076530u, 0x00076531u, 0x00765310u, 0x00076532u, 0x00765320u, 0x00765321u, 0x07653210u,
    0x00007654u, 0x00076540u, 0x00076541u, 0x00765410u, 0x00076542u, 0x00765420u, 0x00765421u, 0x07654210u,
    0x00076543u, 0x00765430u, 0x00765431u, 0x07654310u, 0x00765432u, 0x07654320u, 0x07654321u, 0x76543210u,
};

// Index of the n-th (0-based) set bit of m; n < popc(m), m below 2^32: pick the
// byte by running popcounts, then the bit inside it from the byte table.
__device__ __forceinline__ uint32_t nth_set(uint32_t m, uint32_t n) {
    const uint32_t c0 = __popc(m & 0xFFu);
    const uint32_t c1 = c0 + __popc(m & 0xFF00u);
    const uint32_t c2 = c1 + __popc(m & 0xFF0000u);
    uint32_t b = 0, base = 0;
    if (n >= c0) { b = 8; base = c0; }
    if (n >= c1) { b = 16; base = c1; }
    if (n >= c2) { b = 24; base = c2; }
    const uint32_t rank = (n - base) & 7u;
    return b + ((__ldg(&kSelectInByte[(m >> b) & 0xFFu]) >> (4u * rank)) & 0xFu);
}

// Positions of the set bits of every 12-bit value, 4 bits per rank.  Kernels
// that run playouts copy it into shared memory (32 KB) and pass it to nth_set12.
__device__ const unsigned long long kSelect12[4096] = {
#include "select_tables.inc"
};

// nth_set for masks below 2^24 with the 12-bit table (in shared memory).
__device__ __forceinline__ uint32_t nth_set12(uint32_t m, uint32_t n, const unsigned long long* lut12) {
    const uint32_t c0 = __popc(m & 0xFFFu);
    const bool hi = n >= c0;
    const uint32_t chunk = hi ? (m >> 12) & 0xFFFu : m & 0xFFFu;
    const uint32_t r = (hi ? n - c0 : n) & 15u;
    return (hi ? 12u : 0u) + (uint32_t)((lut12[chunk] >> (4u * r)) & 0xFull);
}

__device__ __forceinline__ void fill_select12(unsigned long long* lut12, uint32_t tid, uint32_t nthr) {
    for (uint32_t e = tid; e < 4096u; e += nthr) lut12[e] = kSelect12[e];
}

// The k lowest set bits of m (k <= popc(m)).
__device__ __forceinline__ uint32_t low_bits(uint32_t m, uint32_t k) {
    if (k == 0) return 0u;
    const uint32_t p = nth_set(m, k - 1);
    return m & (p >= 31 ? 0xFFFFFFFFu : ((2u << p) - 1u));
}

// ------------------------------------------------------------------- state
struct G {
    uint32_t h0, h1, h2, h3;  // hands
    uint32_t rev;
    uint32_t jg0, jg1, jflag;  // joker gaps, white-first flag
    uint32_t cur, drawn, alive, winner;
    uint32_t np, tmask;
    uint32_t mstop;  // 1: cur guessed correctly this turn and may stop (full game tree)

    __device__ __forceinline__ uint32_t hand(uint32_t p) const {
        uint32_t v = h0;
        v = p == 1 ? h1 : v;
        v = p == 2 ? h2 : v;
        v = p == 3 ? h3 : v;
        return v;
    }
    __device__ __forceinline__ void add(uint32_t p, uint32_t bits) {
        h0 |= p == 0 ? bits : 0u;
        h1 |= p == 1 ? bits : 0u;
        h2 |= p == 2 ? bits : 0u;
        h3 |= p == 3 ? bits : 0u;
    }
    __device__ __forceinline__ uint32_t pool() const { return tmask & ~(h0 | h1 | h2 | h3); }
};

// Load a record into registers.  Fields are clamped to their ranges (seats
// 2..4, tiles of the variant, seat indices below the player count) so that a
// malformed record can never index memory out of bounds; valid records pass
// through unchanged.
__device__ __forceinline__ G load_state(const dvc_state& s) {
    G g;
    g.np = (s.nplayers >= 2 && s.nplayers <= 4) ? s.nplayers : 2u;
    g.tmask = s.ntiles >= 26 ? 0x03FFFFFFu : 0x00FFFFFFu;
    g.h0 = s.hand[0] & g.tmask;
    g.h1 = s.hand[1] & g.tmask;
    g.h2 = g.np > 2 ? s.hand[2] & g.tmask : 0u;
    g.h3 = g.np > 3 ? s.hand[3] & g.tmask : 0u;
    g.rev = s.revealed & g.tmask;
    g.jg0 = s.joker_gap[0] <= 24 ? s.joker_gap[0] : 24u;
    g.jg1 = s.joker_gap[1] <= 24 ? s.joker_gap[1] : 24u;
    g.jflag = s.flags & 1u;
    g.mstop = (s.flags >> 1) & 1u;
    g.cur = s.cur < g.np ? s.cur : 0u;
    g.drawn = s.drawn < 26 ? s.drawn : kNone;
    g.alive = s.alive & ((1u << g.np) - 1u);
    g.winner = s.winner < g.np ? s.winner : kNone;
    return g;
}

__device__ __forceinline__ void store_state(const G& g, dvc_state& s) {
    s.hand[0] = g.h0;
    s.hand[1] = g.h1;
    s.hand[2] = g.h2;
    s.hand[3] = g.h3;
    s.revealed = g.rev;
    s.joker_gap[0] = (uint8_t)g.jg0;
    s.joker_gap[1] = (uint8_t)g.jg1;
    s.flags = (uint8_t)(g.jflag | (g.mstop << 1));
    s.cur = (uint8_t)g.cur;
    s.drawn = (uint8_t)g.drawn;
    s.alive = (uint8_t)g.alive;
    s.nplayers = (uint8_t)g.np;
    s.ntiles = g.tmask == 0x03FFFFFFu ? 26 : 24;
    s.winner = (uint8_t)g.winner;
    s.pad[0] = s.pad[1] = s.pad[2] = 0;
}

// Sequence position of joker j (0 black, 1 white) within its owner's hand hp
// (S: any state with the joker fields jg0, jg1, jflag).
template <class S>
__device__ __forceinline__ uint32_t joker_pos(const S& g, uint32_t hp, uint32_t j) {
    const uint32_t gj = j ? g.jg1 : g.jg0, go = j ? g.jg0 : g.jg1;
    const bool other_here = (hp >> (24u + (j ^ 1u))) & 1u;
    // the other joker is first in a shared gap iff (flag ? other is white : other is black)
    const bool other_first = g.jflag ? (j == 0) : (j == 1);
    return gj + ((other_here && (go < gj || (go == gj && other_first))) ? 1u : 0u);
}

// Tile at sequence position s of hand p.
__device__ __forceinline__ uint32_t seq_tile(const G& g, uint32_t p, uint32_t s) {
    const uint32_t hp = g.hand(p);
    const uint32_t jk = hp & kJokerMask;
    if (!jk) return nth_set(hp, s);
    uint32_t before = 0;
#pragma unroll
    for (uint32_t j = 0; j < 2; ++j) {
        if ((jk >> (24u + j)) & 1u) {
            const uint32_t pj = joker_pos(g, hp, j);
            if (pj == s) return 24u + j;
            before += pj < s;
        }
    }
    return nth_set(hp & kNumMask, s - before);
}

// Sequence position of tile t held in hand p.
__device__ __forceinline__ uint32_t seq_pos(const G& g, uint32_t p, uint32_t t) {
    const uint32_t hp = g.hand(p);
    if (t >= 24u) return joker_pos(g, hp, t - 24u);
    const uint32_t k = __popc(hp & kNumMask & ((1u << t) - 1u));
    uint32_t pos = k;
    if ((hp >> 24) & 1u) pos += g.jg0 <= k;
    if ((hp >> 25) & 1u) pos += g.jg1 <= k;
    return pos;
}

// Tile in the h-th face-down slot (left to right) of the hand with tiles hp.
template <class S>
__device__ __forceinline__ uint32_t hidden_in(const S& g, uint32_t hp, uint32_t h) {
    const uint32_t hid = hp & ~g.rev;
    const uint32_t hj = hid & kJokerMask;
    const uint32_t hn = hid & kNumMask;
    if (!hj) return nth_set(hn, h);
    // face-down index of each face-down joker
    uint32_t idx[2] = {0xFFu, 0xFFu};
#pragma unroll
    for (uint32_t j = 0; j < 2; ++j) {
        if ((hj >> (24u + j)) & 1u) {
            const uint32_t gj = j ? g.jg1 : g.jg0;
            uint32_t n = __popc(hn & low_bits(hp & kNumMask, gj));
            const uint32_t o = j ^ 1u;
            if ((hj >> (24u + o)) & 1u) n += joker_pos(g, hp, o) < joker_pos(g, hp, j);
            idx[j] = n;
        }
    }
    if (idx[0] == h) return 24u;
    if (idx[1] == h) return 25u;
    const uint32_t skip = (idx[0] < h) + (idx[1] < h);
    return nth_set(hn, h - skip);
}

// Tile in the h-th face-down slot (left to right) of hand p.
__device__ __forceinline__ uint32_t hidden_slot(const G& g, uint32_t p, uint32_t h) {
    return hidden_in(g, g.hand(p), h);
}

// The joker-gap part of a sorted insertion of tile t into the hand with
// tiles hp (before t is added); a joker takes one word for its position.
template <class S, class R>
__device__ __forceinline__ void insert_gaps(S& g, uint32_t hp, uint32_t t, R& r) {
    if (t < 24u) {
        const uint32_t k = __popc(hp & kNumMask & ((1u << t) - 1u));
        if ((hp >> 24) & 1u) g.jg0 += g.jg0 > k;
        if ((hp >> 25) & 1u) g.jg1 += g.jg1 > k;
    } else {
        const uint32_t j = t - 24u, o = j ^ 1u;
        const uint32_t pos = pick(r.next(), __popc(hp) + 1u);
        uint32_t gap = pos, flag = 0u;
        if ((hp >> (24u + o)) & 1u) {
            const uint32_t po = joker_pos(g, hp, o);
            const bool new_first = pos <= po;
            gap = new_first ? pos : pos - 1u;
            const uint32_t go = o ? g.jg1 : g.jg0;
            if (gap == go) flag = (new_first ? j : o) == 1u ? 1u : 0u;
        }
        if (j) g.jg1 = gap; else g.jg0 = gap;
        g.jflag = flag;
    }
}

// Sorted insertion of tile t into hand p (Sec. II-A).  Numbered: immediately
// before the first larger numbered tile, so jokers of that gap stay left.
// Joker: uniform over the len+1 insertion points (one word).
template <class R>
__device__ __forceinline__ void insert_tile(G& g, uint32_t p, uint32_t t, R& r) {
    insert_gaps(g, g.hand(p), t, r);
    g.add(p, 1u << t);
}

template <class R>
__device__ __forceinline__ void draw(G& g, R& r) {
    const uint32_t pool = g.pool();
    if (!pool) {
        g.drawn = kNone;
        return;
    }
    const uint32_t t = nth_set(pool, pick(r.next(), __popc(pool)));
    insert_tile(g, g.cur, t, r);
    g.drawn = t;
}

__device__ __forceinline__ uint32_t next_alive(uint32_t alive, uint32_t cur, uint32_t np) {
    const uint32_t dup = alive | (alive << np);
    const uint32_t m = dup >> (cur + 1u);
    const uint32_t q = cur + (uint32_t)__ffs(m);
    return q >= np ? q - np : q;
}

enum : int { kTurnOver = 0, kGuessAgain = 1, kGameOver = 2 };

// Resolve guess `x` at the tile `target` of seat q (Sec. II-A).  In a playout
// a correct guess continues iff the next word < cont_thr; in the tree it ends
// the turn (Sec. III-A, simplification 2).
template <class R>
__device__ __forceinline__ int resolve(G& g, uint32_t q, uint32_t target, uint32_t x, bool in_tree, uint32_t cont_thr,
                                       R& r) {
    if (x == target) {
        g.rev |= 1u << target;
        if (!(g.hand(q) & ~g.rev)) g.alive &= ~(1u << q);
        if (__popc(g.alive) == 1) {
            g.winner = g.cur;
            return kGameOver;
        }
        if (!in_tree && cont_thr != 0u && r.next() < cont_thr) return kGuessAgain;
        return kTurnOver;
    }
    const uint32_t c = g.cur;
    const uint32_t t = g.drawn != kNone ? g.drawn : hidden_slot(g, c, 0);
    g.rev |= 1u << t;
    if (!(g.hand(c) & ~g.rev)) g.alive &= ~(1u << c);
    if (__popc(g.alive) == 1) {
        g.winner = (uint32_t)__ffs(g.alive) - 1u;
        return kGameOver;
    }
    return kTurnOver;
}

template <class R>
__device__ __forceinline__ void next_turn(G& g, R& r) {
    g.cur = next_alive(g.alive, g.cur, g.np);
    draw(g, r);
}

// floor(k / n) for k < 4096 and 1 <= n <= 31 from magic[n] = floor((2^32-1)/n) + 1:
// k * magic / 2^32 exceeds k/n by less than 2^-20 < 1/n, so the floor is exact.
__device__ __forceinline__ uint32_t div_small(uint32_t k, uint32_t n, const uint32_t* magic) {
    if (magic == nullptr) return k / n;
    return n == 1u ? k : __umulhi(k, magic[n]);
}

__device__ __forceinline__ void fill_magic(uint32_t* magic, uint32_t tid, uint32_t nthr) {
    for (uint32_t n = tid; n < 32u; n += nthr) magic[n] = n < 2u ? 0u : 0xFFFFFFFFu / n + 1u;
}

// A uniform random guess among the legal ones (canonical order: opponents
// from cur+1, face-down slots left to right, identities ascending; the set is
// the product of face-down slots and identities outside own hand and face-up).
// The guess (slot s, identity index i) is correct iff i is the rank of the
// slot's tile among the unknown identities, so only one select is needed.
template <class R>
__device__ __forceinline__ int random_guess(G& g, R& r, uint32_t cont_thr, const uint32_t* magic = nullptr) {
    const uint32_t U = g.tmask & ~g.hand(g.cur) & ~g.rev;
    const uint32_t nid = __popc(U);
    uint32_t cnt[3], qs[3], nslots = 0;
#pragma unroll
    for (uint32_t off = 1; off < 4; ++off) {
        uint32_t q = g.cur + off;
        q = q >= g.np ? q - g.np : q;
        const uint32_t c = (off < g.np) ? __popc(g.hand(q) & ~g.rev) : 0u;
        cnt[off - 1] = c;
        qs[off - 1] = q;
        nslots += c;
    }
    const uint32_t k = pick(r.next(), nslots * nid);
    uint32_t s = div_small(k, nid, magic);
    const uint32_t i = k - s * nid;
    uint32_t q = qs[0];
    if (s >= cnt[0]) {
        s -= cnt[0];
        q = qs[1];
        if (s >= cnt[1]) {
            s -= cnt[1];
            q = qs[2];
        }
    }
    const uint32_t target = hidden_slot(g, q, s);
    const uint32_t rank = __popc(U & ((1u << target) - 1u));
    return resolve(g, q, target, rank == i ? target : 0xFFu, false, cont_thr, r);
}

// The identities the ordering-aware playout policy keeps for the face-down
// slot of player q that holds tile t: unknown numbered identities strictly
// between the nearest face-up numbered tiles to the slot's left and right in
// q's row (by id), and every unknown joker.  For a numbered t the row's
// numbered tiles below t are exactly those to its left; a joker stands after
// the first joker_gap numbered tiles.
__device__ __forceinline__ uint32_t ordered_fit(const G& g, uint32_t q, uint32_t t, uint32_t U) {
    const uint32_t hn = g.hand(q) & kNumMask;
    const uint32_t left = t < 24u ? hn & ((1u << t) - 1u) : low_bits(hn, t == 24u ? g.jg0 : g.jg1);
    const uint32_t lrev = left & g.rev, rrev = hn & ~left & ~(t < 24u ? 1u << t : 0u) & g.rev;
    const uint32_t lo_mask = lrev ? (2u << (31 - __clz(lrev))) - 1u : 0u;       // identities <= left neighbour
    const uint32_t hi_mask = rrev ? (1u << (__ffs(rrev) - 1)) - 1u : kNumMask;  // identities < right neighbour
    return (U & kNumMask & hi_mask & ~lo_mask) | (U & kJokerMask);
}

// A uniform random guess under the ordering-aware playout policy (not the
// paper's: a stronger playout to compare with).  Same canonical order and one
// word per guess, restricted per slot by ordered_fit.
template <class R>
__device__ __forceinline__ int random_guess_ordered(G& g, R& r, uint32_t cont_thr) {
    const uint32_t U = g.tmask & ~g.hand(g.cur) & ~g.rev;
    uint32_t total = 0;
    for (uint32_t off = 1; off < g.np; ++off) {
        uint32_t q = g.cur + off;
        q = q >= g.np ? q - g.np : q;
        if (!((g.alive >> q) & 1u)) continue;
        const uint32_t nh = __popc(g.hand(q) & ~g.rev);
        for (uint32_t h = 0; h < nh; ++h) total += __popc(ordered_fit(g, q, hidden_slot(g, q, h), U));
    }
    uint32_t k = pick(r.next(), total);
    for (uint32_t off = 1; off < g.np; ++off) {
        uint32_t q = g.cur + off;
        q = q >= g.np ? q - g.np : q;
        if (!((g.alive >> q) & 1u)) continue;
        const uint32_t nh = __popc(g.hand(q) & ~g.rev);
        for (uint32_t h = 0; h < nh; ++h) {
            const uint32_t t = hidden_slot(g, q, h);
            const uint32_t F = ordered_fit(g, q, t, U);
            const uint32_t c = __popc(F);
            if (k < c) {
                const uint32_t x = nth_set(F, k);
                return resolve(g, q, t, x == t ? t : 0xFFu, false, cont_thr, r);
            }
            k -= c;
        }
    }
    return resolve(g, g.cur, 0u, 0xFFu, false, cont_thr, r);  // unreachable: total counts every kept guess
}

// One playout to the end (Sec. II-B); returns the winner.  Every guess turns
// one tile face up, so a game has at most 26 guesses; the cap only stops a
// malformed record (result kNone, credited to nobody).
template <class R>
__device__ __forceinline__ uint32_t playout(G g, R& r, uint32_t cont_thr, const uint32_t* magic = nullptr) {
    for (int guard = 0; guard < 128; ++guard) {
        const int res = random_guess(g, r, cont_thr, magic);
        if (res == kGameOver) return g.winner;
        if (res == kTurnOver) next_turn(g, r);
    }
    return kNone;
}

// The playout state with hands held relative to the mover: a0 is the hand of
// seat cur, a1, a2, a3 those of seats cur + 1, cur + 2, cur + 3 (modulo np);
// positions from np on hold 0.  The opponents are then visited in the
// canonical order (from cur + 1) with no selection of hands by seat, and a
// new turn rotates the four words once.  alive and winner stay by seat.
struct GR {
    uint32_t a0, a1, a2, a3;
    uint32_t rev, jg0, jg1, jflag;
    uint32_t cur, drawn, alive, winner, np, tmask;
};

__device__ __forceinline__ GR to_gr(const G& g) {
    GR r;
    uint32_t q1 = g.cur + 1u, q2 = g.cur + 2u, q3 = g.cur + 3u;
    q1 = q1 >= g.np ? q1 - g.np : q1;
    q2 = q2 >= g.np ? q2 - g.np : q2;
    q3 = q3 >= g.np ? q3 - g.np : q3;
    r.a0 = g.hand(g.cur);
    r.a1 = g.hand(q1);
    r.a2 = g.np > 2u ? g.hand(q2) : 0u;
    r.a3 = g.np > 3u ? g.hand(q3) : 0u;
    r.rev = g.rev;
    r.jg0 = g.jg0;
    r.jg1 = g.jg1;
    r.jflag = g.jflag;
    r.cur = g.cur;
    r.drawn = g.drawn;
    r.alive = g.alive;
    r.winner = g.winner;
    r.np = g.np;
    r.tmask = g.tmask;
    return r;
}

// One playout step in the relative form: random_guess, then next_turn if the
// turn passes -- the same rules, the same words in the same order.
template <class R>
__device__ __forceinline__ int step_gen(GR& g, R& r, uint32_t cont_thr, const uint32_t* magic) {
    r.ensure(4);
    // the guess: opponent slots in canonical order times unknown identities
    const uint32_t U = g.tmask & ~g.a0 & ~g.rev;
    const uint32_t nid = __popc(U);
    const uint32_t c1 = __popc(g.a1 & ~g.rev), c2 = __popc(g.a2 & ~g.rev), c3 = __popc(g.a3 & ~g.rev);
    const uint32_t k = pick(r.next(), (c1 + c2 + c3) * nid);
    uint32_t s = div_small(k, nid, magic);
    const uint32_t i = k - s * nid;
    uint32_t off = 1u, hq = g.a1;
    if (s >= c1) {
        s -= c1;
        off = 2u;
        hq = g.a2;
        if (s >= c2) {
            s -= c2;
            off = 3u;
            hq = g.a3;
        }
    }
    const uint32_t target = hidden_in(g, hq, s);
    const uint32_t tb = 1u << target;
    if (__popc(U & (tb - 1u)) == i) {  // correct: the target is revealed
        g.rev |= tb;
        if (!(hq & ~g.rev)) {
            uint32_t q = g.cur + off;
            q = q >= g.np ? q - g.np : q;
            g.alive &= ~(1u << q);
        }
        if (__popc(g.alive) == 1) {
            g.winner = g.cur;
            return kGameOver;
        }
        if (cont_thr != 0u && r.next() < cont_thr) return kGuessAgain;
    } else {  // wrong: the mover reveals its drawn tile, else its leftmost face-down one
        uint32_t t = g.drawn;
        if (t == kNone) {  // the leftmost face-down tile: the lowest one unless a joker is face down
            const uint32_t hid = g.a0 & ~g.rev;
            t = (hid & kJokerMask) ? hidden_in(g, g.a0, 0u) : (uint32_t)__ffs(hid) - 1u;
        }
        g.rev |= 1u << t;
        if (!(g.a0 & ~g.rev)) g.alive &= ~(1u << g.cur);
        if (__popc(g.alive) == 1) {
            g.winner = (uint32_t)__ffs(g.alive) - 1u;
            return kGameOver;
        }
    }
    // the next live seat moves: rotate the hands by d = its distance (1 .. np-1)
    const uint32_t nc = next_alive(g.alive, g.cur, g.np);
    const uint32_t d = nc > g.cur ? nc - g.cur : nc + g.np - g.cur;
    if (g.np == 4u) {
        if (d & 1u) {
            const uint32_t t = g.a0;
            g.a0 = g.a1;
            g.a1 = g.a2;
            g.a2 = g.a3;
            g.a3 = t;
        }
        if (d & 2u) {
            uint32_t t = g.a0;
            g.a0 = g.a2;
            g.a2 = t;
            t = g.a1;
            g.a1 = g.a3;
            g.a3 = t;
        }
    } else if (g.np == 3u) {
        const uint32_t b0 = d == 1u ? g.a1 : g.a2, b1 = d == 1u ? g.a2 : g.a0, b2 = d == 1u ? g.a0 : g.a1;
        g.a0 = b0;
        g.a1 = b1;
        g.a2 = b2;
    } else {
        const uint32_t t = g.a0;
        g.a0 = g.a1;
        g.a1 = t;
    }
    g.cur = nc;
    // ... and draws
    const uint32_t pool = g.tmask & ~(g.a0 | g.a1 | g.a2 | g.a3);
    if (!pool) {
        g.drawn = kNone;
        return kTurnOver;
    }
    const uint32_t t = nth_set(pool, pick(r.next(), __popc(pool)));
    insert_gaps(g, g.a0, t, r);
    g.a0 |= 1u << t;
    g.drawn = t;
    return kTurnOver;
}

// Words for the playout loop of the pooled kernel: a short queue that is
// topped up once, at the start of each game step, with enough words for the
// whole step (a guess, a continue coin, a draw and a joker position at most),
// so the step itself never branches to refill.
struct WordQueue {
    uint32_t k0, k1, blk, j, i, tw;
    uint32_t q0, q1, q2, q3, q4, q5, q6;
    uint32_t left;

    __device__ __forceinline__ void open(uint64_t seed, uint32_t tree, uint32_t jj, uint32_t ii, uint32_t tag) {
        k0 = (uint32_t)seed;
        k1 = tree;
        blk = 0;
        j = jj;
        i = ii;
        tw = tag + 16u * (uint32_t)(seed >> 32);
        left = 0;
    }
    // make at least n (<= 4) words available
    __device__ __forceinline__ void ensure(uint32_t n) {
        if (left >= n) return;
        uint32_t a = blk, b = j, c = i, d = tw;
        philox10(a, b, c, d, k0, k1);
        ++blk;
        // append a, b, c, d after the `left` words already queued (left <= 3)
        q0 = left == 0 ? a : q0;
        q1 = left == 0 ? b : (left == 1 ? a : q1);
        q2 = left == 0 ? c : (left == 1 ? b : (left == 2 ? a : q2));
        q3 = left == 0 ? d : (left == 1 ? c : (left == 2 ? b : a));
        q4 = left == 1 ? d : (left == 2 ? c : b);
        q5 = left == 2 ? d : c;
        q6 = d;
        left += 4;
    }
    __device__ __forceinline__ uint32_t next() {
        const uint32_t r = q0;
        q0 = q1;
        q1 = q2;
        q2 = q3;
        q3 = q4;
        q4 = q5;
        q5 = q6;
        --left;
        return r;
    }
    // words handed out so far
    __device__ __forceinline__ uint32_t used() const { return 4u * blk - left; }
};

// The same stream as WordQueue, queued in shared memory: a ring of 16 words
// per thread, word s of thread t at ring[s * stride + t] (a warp's lanes hit
// consecutive banks).  Refills are warp-wide: when any lane is short of words,
// every lane with room for a block appends its next Philox block, so one
// evaluation of the Philox rounds serves most lanes of the warp instead of
// the few that ran dry.  Word order per stream is unchanged.
struct RingQueue {
    uint32_t* ring;  // &ring[threadIdx.x]
    uint32_t stride;
    uint32_t k0, k1, j, i, tw;
    uint32_t head, tail;  // words handed out / appended (tail = 4 x blocks)

    __device__ __forceinline__ void open(uint64_t seed, uint32_t tree, uint32_t jj, uint32_t ii, uint32_t tag) {
        k0 = (uint32_t)seed;
        k1 = tree;
        j = jj;
        i = ii;
        tw = tag + 16u * (uint32_t)(seed >> 32);
        head = tail = 0u;
    }
    // make at least n (<= 4) words available; called by converged lanes
    __device__ __forceinline__ void ensure(uint32_t n) {
        const uint32_t left = tail - head;
        if (__any_sync(__activemask(), left < n) && left <= 12u) {
            uint32_t a = tail >> 2, b = j, c = i, d = tw;
            philox10(a, b, c, d, k0, k1);
            const uint32_t s = tail & 15u;  // tail is a multiple of 4: slots s..s+3 do not wrap
            ring[s * stride] = a;
            ring[(s + 1u) * stride] = b;
            ring[(s + 2u) * stride] = c;
            ring[(s + 3u) * stride] = d;
            tail += 4u;
        }
    }
    __device__ __forceinline__ uint32_t next() {
        const uint32_t r = ring[(head & 15u) * stride];
        ++head;
        return r;
    }
    __device__ __forceinline__ uint32_t used() const { return head; }
    // Continue a stream another lane started (stream fields already set):
    // h words were handed out; this lane's ring gets the block holding word
    // h, so the next word is word h of the stream.
    __device__ __forceinline__ void resume(uint32_t h) {
        head = h;
        tail = h & ~3u;
        uint32_t a = tail >> 2, b = j, c = i, d = tw;
        philox10(a, b, c, d, k0, k1);
        const uint32_t s = tail & 15u;
        ring[s * stride] = a;
        ring[(s + 1u) * stride] = b;
        ring[(s + 2u) * stride] = c;
        ring[(s + 3u) * stride] = d;
        tail += 4u;
    }
};

// One step of a two-player, 24-tile playout (no jokers): the mover guesses;
// a correct guess reveals the tile and either ends the game, grants another
// guess (continue coin) or passes the turn; a wrong guess reveals the mover's
// drawn tile (or lowest face-down tile) and passes the turn; the next mover
// draws.  Same rules and same word order as random_guess + next_turn.
template <class Q>
__device__ __forceinline__ int step_2p24(uint32_t& h0, uint32_t& h1, uint32_t& rev, uint32_t& cur, uint32_t& drawn,
                                         uint32_t& winner, Q& r, uint32_t cont_thr, const uint32_t* magic,
                                         const unsigned long long* lut12) {
    r.ensure(3);
    const uint32_t hc = cur ? h1 : h0;
    const uint32_t hidq = (cur ? h0 : h1) & ~rev;
    const uint32_t U = kNumMask & ~hc & ~rev;
    const uint32_t nid = __popc(U);
    const uint32_t k = __umulhi(r.next(), __popc(hidq) * nid);
    const uint32_t s = div_small(k, nid, magic);
    const uint32_t i = k - s * nid;
    const uint32_t target = nth_set12(hidq, s, lut12);
    if (__popc(U & ((1u << target) - 1u)) == i) {
        rev |= 1u << target;
        if (hidq == (1u << target)) {
            winner = cur;
            return kGameOver;
        }
        if (cont_thr != 0u && r.next() < cont_thr) return kGuessAgain;
    } else {
        const uint32_t t = drawn != kNone ? drawn : (uint32_t)__ffs(hc & ~rev) - 1u;
        rev |= 1u << t;
        if (!(hc & ~rev)) {
            winner = cur ^ 1u;
            return kGameOver;
        }
    }
    cur ^= 1u;
    const uint32_t pool = kNumMask & ~(h0 | h1);
    if (pool) {
        const uint32_t t = nth_set12(pool, __umulhi(r.next(), __popc(pool)), lut12);
        if (cur) h1 |= 1u << t;
        else h0 |= 1u << t;
        drawn = t;
    } else {
        drawn = kNone;
    }
    return kTurnOver;
}

// step_2p24 under the ordering-aware playout policy: the guess is uniform
// over the (face-down slot, identity) pairs the policy keeps.  Without
// jokers a row is in id order, so a slot's face-up neighbours are the
// opponent's face-up tiles just below and just above its tile.
template <class Q>
__device__ __forceinline__ int step_2p24_ordered(uint32_t& h0, uint32_t& h1, uint32_t& rev, uint32_t& cur,
                                                 uint32_t& drawn, uint32_t& winner, Q& r, uint32_t cont_thr,
                                                 const unsigned long long* lut12) {
    r.ensure(3);
    const uint32_t hc = cur ? h1 : h0, hq = cur ? h0 : h1;
    const uint32_t hidq = hq & ~rev, rq = hq & rev;
    const uint32_t U = kNumMask & ~hc & ~rev;
    auto fit = [&](uint32_t t) {
        const uint32_t below = rq & ((1u << t) - 1u), above = rq & ~((2u << t) - 1u);
        const uint32_t lo_mask = below ? (2u << (31 - __clz(below))) - 1u : 0u;
        const uint32_t hi_mask = above ? (1u << (__ffs(above) - 1)) - 1u : kNumMask;
        return U & hi_mask & ~lo_mask;
    };
    uint32_t total = 0;
    for (uint32_t m = hidq; m; m &= m - 1u) total += __popc(fit(__ffs(m) - 1u));
    uint32_t k = __umulhi(r.next(), total), target = 0u, x = 0u;
    for (uint32_t m = hidq; m; m &= m - 1u) {
        const uint32_t t = __ffs(m) - 1u, F = fit(t), c = __popc(F);
        if (k < c) {
            target = t;
            x = nth_set12(F, k, lut12);
            break;
        }
        k -= c;
    }
    if (x == target) {
        rev |= 1u << target;
        if (hidq == (1u << target)) {
            winner = cur;
            return kGameOver;
        }
        if (cont_thr != 0u && r.next() < cont_thr) return kGuessAgain;
    } else {
        const uint32_t t = drawn != kNone ? drawn : (uint32_t)__ffs(hc & ~rev) - 1u;
        rev |= 1u << t;
        if (!(hc & ~rev)) {
            winner = cur ^ 1u;
            return kGameOver;
        }
    }
    cur ^= 1u;
    const uint32_t pool = kNumMask & ~(h0 | h1);
    if (pool) {
        const uint32_t t = nth_set12(pool, __umulhi(r.next(), __popc(pool)), lut12);
        if (cur) h1 |= 1u << t;
        else h0 |= 1u << t;
        drawn = t;
    } else {
        drawn = kNone;
    }
    return kTurnOver;
}

// The first step of a two-player 24-tile playout that begins where the mover
// may stop (winner == kPend): the continue coin; on "stop" the turn passes
// and the next mover draws, on "go on" the next step is an ordinary guess.
template <class Q>
__device__ __forceinline__ int step_2p24_pending(uint32_t& h0, uint32_t& h1, uint32_t& cur, uint32_t& drawn,
                                                 uint32_t& winner, Q& r, uint32_t cont_thr,
                                                 const unsigned long long* lut12) {
    r.ensure(2);
    winner = kNone;
    if (cont_thr != 0u && r.next() < cont_thr) return kGuessAgain;
    cur ^= 1u;
    const uint32_t pool = kNumMask & ~(h0 | h1);
    if (pool) {
        const uint32_t t = nth_set12(pool, __umulhi(r.next(), __popc(pool)), lut12);
        if (cur) h1 |= 1u << t;
        else h0 |= 1u << t;
        drawn = t;
    } else {
        drawn = kNone;
    }
    return kTurnOver;
}

// Is action (q, slot s, identity x) legal for the seat to move?
__device__ __forceinline__ bool guess_legal(const G& g, uint32_t q, uint32_t s, uint32_t x) {
    if (q == g.cur || q >= g.np || !((g.alive >> q) & 1u)) return false;
    const uint32_t hq = g.hand(q);
    if (s >= (uint32_t)__popc(hq)) return false;
    if ((g.rev >> seq_tile(g, q, s)) & 1u) return false;
    if (!((g.tmask >> x) & 1u)) return false;
    if (((g.hand(g.cur) | g.rev) >> x) & 1u) return false;
    return true;
}

// Is `code` a legal action for the seat to move: STOP when it may stop, or a
// legal guess?
__device__ __forceinline__ bool action_legal(const G& g, uint32_t code) {
    if (code == kStop) return g.mstop != 0u;
    return guess_legal(g, code >> 10, (code >> 5) & 31u, code & 31u);
}

// In-tree transition (and self-play move) for an action: STOP passes the
// turn; a guess is resolved with no playout coin, and after a correct guess
// that does not end the game the player keeps the turn and may stop when
// cont is set (the full game tree of Fig. 2a), else the turn passes; when it
// passes, the next seat draws on the tree stream.
__device__ __forceinline__ void tree_apply(G& g, uint32_t code, Rng& tr, bool cont = false) {
    if (code == kStop) {
        g.mstop = 0u;
        next_turn(g, tr);
        return;
    }
    const uint32_t q = code >> 10, s = (code >> 5) & 31u, x = code & 31u;
    const uint32_t target = seq_tile(g, q, s);
    if (resolve(g, q, target, x, true, 0u, tr) == kGameOver) {
        g.mstop = 0u;
        return;
    }
    if (cont && target == x) {
        g.mstop = 1u;
        return;
    }
    g.mstop = 0u;
    next_turn(g, tr);
}

// Canonical rank of an action at a node whose mover is cur: STOP first, then
// guesses by opponent (from cur + 1), slot, identity.
__device__ __forceinline__ uint32_t canon_rank(uint32_t code, uint32_t cur, uint32_t np) {
    if (code == kStop) return 0u;
    const uint32_t q = code >> 10;
    uint32_t d = q + np - cur - 1u;
    d = d >= np ? d - np : d;
    return 1u + ((d << 10) | (code & 1023u));
}

// A playout that starts where the mover may stop first draws the continue
// coin (a playout guesses again after a correct guess iff the next word is
// below cont_thr).
template <class R>
__device__ __forceinline__ void playout_begin(G& g, R& r, uint32_t cont_thr) {
    if (!g.mstop || g.winner != kNone) return;
    g.mstop = 0u;
    r.ensure(4);
    if (!(cont_thr != 0u && r.next() < cont_thr)) next_turn(g, r);
}

// ------------------------------------------------------------------- UCT
// ln(x), x >= 1, in IEEE single precision: x = m 2^e with m in
// [sqrt(1/2), sqrt(2)); ln x = e ln2 + 2 atanh(z), z = (m-1)/(m+1), by the
// atanh series up to z^11 in Horner form (|z| <= 0.1716: the next term is
// below 2^-30 of the sum).  Every operation is an explicitly rounded IEEE
// float op (no contraction); ln2 is the float nearest to it.
__device__ __forceinline__ float ln_series(float x) {
    const uint32_t bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    if (m > 1.41421354f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float z = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float z2 = __fmul_rn(z, z);
    // 1/(2k+1) as compile-time constants: the compiler rounds each quotient
    // correctly, exactly as the runtime IEEE division would
    constexpr float inv[6] = {1.0f / 1.0f, 1.0f / 3.0f, 1.0f / 5.0f, 1.0f / 7.0f, 1.0f / 9.0f, 1.0f / 11.0f};
    float p = inv[5];
#pragma unroll
    for (int k = 4; k >= 0; --k) p = __fadd_rn(__fmul_rn(p, z2), inv[k]);
    const float lnm = __fmul_rn(2.0f, __fmul_rn(z, p));
    return __fadd_rn(__fmul_rn((float)e, 0.693147182f), lnm);
}

}  // namespace dvc
