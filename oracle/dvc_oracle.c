/*
 * dvc_oracle.c -- CPU oracle for the Da Vinci Code Monte Carlo Tree Search of
 * arXiv 2403.10720 ("Development and Application of a Monte Carlo Tree Search
 * Algorithm for Simulating Da Vinci Code Game Strategies").
 *
 * TEST INFRASTRUCTURE.  This is the plain, slow, single-threaded statement of
 * what the GPU engine computes.  Only the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg load it; the product path never does.
 * It shares no code, header, table or helper with the CUDA library: hands are
 * explicit left-to-right tile sequences here (the GPU keeps bitmasks), every
 * choice is made by building the full candidate list in canonical order and
 * indexing it, and Philox is restated from its published definition.
 *
 * Passages followed (paper sections):
 *   rules of the game ............ Sec. II-A (tile set, deal, draw + sorted
 *                                  insertion, guess, correct guess -> reveal and
 *                                  optional extra guess, wrong guess -> reveal
 *                                  the drawn tile, last player standing wins)
 *   random playout ............... Sec. II-B (game played out by random choices)
 *   node = (position, number) .... Sec. III-A, simplification 1
 *   plausible numbers sampled .... Sec. III-A (determinization per simulation)
 *   stop after a correct guess ... Sec. III-A, simplification 2 (inside the tree)
 *   expansion depth limit ........ Sec. III-A, simplification 3
 *   plausible-set nodes (vanilla)  Sec. III-A, the tree simplification 1 removes
 *   continue / stop nodes ........ Fig. 2a, the tree simplification 2 removes
 *   root-parallel merge .......... Sec. III-B
 *   Philox-4x32-10 ............... Salmon, Moraes, Dror, Shaw, "Parallel Random
 *                                  Numbers: As Easy as 1, 2, 3", SC'11
 *   ln for UCT (float) ........... argument reduction to [sqrt(1/2), sqrt(2))
 *                                  and ln m = 2 atanh((m-1)/(m+1)) by its
 *                                  Taylor series (classic Cody-Waite style)
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vectors; ln against libm;
 * rule invariants on traced playouts; the 88-guess root count of Sec. III-A;
 * a closed-form 1/k endgame; exact win probabilities of tiny endgames by an
 * independent exhaustive enumerator; determinizer counts against brute-force
 * enumeration plus a chi-square test; UCB1 selection on a forced-win toy tree;
 * visit-count invariants; the full game tree's STOP action and kept turn; the
 * ordering-aware policy against the enumerator; vanilla MCTS-dvc's set layer
 * against the determinizer's samples.  The value-network functions are pinned
 * by finite differences and by a closed-form single-layer case.
 *
 * Where the paper leaves a point open, the reading taken is stated beside the
 * code it shapes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NUMBERED 24          /* tiles 0..23: value v = t/2, colour c = t%2 */
#define JOKER_BLACK 24
#define JOKER_WHITE 25
#define MAXT 26
#define MAXP 4
#define MAXLEGAL (3 * MAXT * MAXT)

enum { TAG_INIT = 1, TAG_DET = 2, TAG_TREE = 3, TAG_ROLL = 4, TAG_PLAY = 5 };

/* STOP (Fig. 2a): end a turn after a correct guess; the first of a node's
 * actions in canonical order.  Guesses are coded seat << 10 | slot << 5 |
 * identity. */
enum { STOP = 0xFFF };

/* SET: a plausible-number-set node of vanilla MCTS-dvc (Sec. III-A): a child
 * of the root standing for one assignment of the tiles the observer cannot
 * see. */
enum { SET = 0xFFE };

typedef struct {
    int32_t nplayers, ntiles, deal, max_predraw, max_revealed;
    uint32_t cont_thr; /* after a correct guess in a playout: guess again iff word < cont_thr; 0 = never, no word */
    double c_uct;
    int32_t d_max, playouts;
    int32_t policy; /* playout guesses: 0 uniform over the legal guesses; 1 ordering-aware (see legal_list_policy) */
    int32_t tree_continue; /* in the tree: 0 a correct guess ends the turn (Sec. III-A); 1 the player may go on (Fig. 2a) */
    int32_t vanilla; /* 1: the root's children are plausible-number sets (vanilla MCTS-dvc, Sec. III-A) */
} or_config;

/* ------------------------------------------------------------------ Philox */

/* Philox-4x32 with 10 rounds (Salmon et al., SC'11): each round multiplies
 * words 0 and 2 by fixed odd constants, swaps the halves, and xors in the
 * round key; the key is bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One random stream: key = (low word of seed, tree id), counter =
 * (block, playout, iteration or leaf, tag + 16 * high word of seed).
 * Words of a block are used in order, then the block index advances. */
typedef struct {
    uint32_t key[2], ctr[4], buf[4];
    int used;
    int64_t words; /* words consumed so far (statistics only) */
} stream;

static void stream_open(stream* s, uint64_t seed, uint32_t tree, uint32_t j, uint32_t i, uint32_t tag) {
    s->key[0] = (uint32_t)seed;
    s->key[1] = tree;
    s->ctr[0] = 0;
    s->ctr[1] = j;
    s->ctr[2] = i;
    s->ctr[3] = tag + 16u * (uint32_t)(seed >> 32);
    s->used = 4;
    s->words = 0;
}

static uint32_t next_word(stream* s) {
    if (s->used == 4) {
        or_philox4x32_10(s->ctr, s->key, s->buf);
        s->ctr[0]++;
        s->used = 0;
    }
    s->words++;
    return s->buf[s->used++];
}

/* A uniform choice among n candidates from one 32-bit word: floor(w*n/2^32). */
static int pick(uint32_t w, int n) { return (int)(((uint64_t)w * (uint64_t)n) >> 32); }

/* A choice among W candidates from a 64-bit value r: floor(r*W/2^64). */
static uint64_t pick64(uint64_t r, uint64_t W) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)W) >> 64);
}

static uint64_t next_word64(stream* s) {
    uint64_t lo = next_word(s);
    uint64_t hi = next_word(s);
    return (hi << 32) | lo;
}

/* ------------------------------------------------------------------- state */

typedef struct {
    int P, T;
    int seq[MAXP][MAXT]; /* each hand left to right */
    int len[MAXP];
    int rev[MAXT];   /* 1 = face up */
    int owner[MAXT]; /* -1 = in the pool */
    int alive[MAXP];
    int cur, drawn, winner; /* drawn: tile drawn this turn or -1; winner -1 while running */
    int mstop;              /* 1: cur has guessed correctly this turn and may stop or guess again */
} ost;

/* Boundary format (32 bytes, little endian): hand[4] u32 tile bitmasks at 0,
 * revealed u32 at 16, joker gaps u8[2] at 20 (numbered tiles left of each
 * joker in its owner's hand, 0 when in the pool), flags u8 at 22 (bit 0: both
 * jokers share an owner and a gap and the white one is first; bit 1: the
 * player to move has guessed correctly this turn and may stop), cur at 23,
 * drawn at 24 (0xFF none), alive mask at 25, players at 26, tiles at 27,
 * winner at 28 (0xFF while running), zero padding 29..31. */
static uint32_t rd32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static void wr32(uint8_t* p, uint32_t v) {
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}

static int numbered_before(const ost* s, int p, int pos) {
    int n = 0;
    for (int i = 0; i < pos; i++) n += s->seq[p][i] < NUMBERED;
    return n;
}

static void pack(const ost* s, uint8_t* out) {
    memset(out, 0, 32);
    for (int p = 0; p < s->P; p++) {
        uint32_t m = 0;
        for (int i = 0; i < s->len[p]; i++) m |= 1u << s->seq[p][i];
        wr32(out + 4 * p, m);
    }
    uint32_t rv = 0;
    for (int t = 0; t < s->T; t++) if (s->rev[t]) rv |= 1u << t;
    wr32(out + 16, rv);
    int jpos[2] = {-1, -1}, jown[2] = {-1, -1};
    for (int j = 0; j < 2; j++) {
        int t = JOKER_BLACK + j;
        if (t >= s->T || s->owner[t] < 0) continue;
        int p = s->owner[t];
        for (int i = 0; i < s->len[p]; i++) if (s->seq[p][i] == t) jpos[j] = i;
        jown[j] = p;
        out[20 + j] = (uint8_t)numbered_before(s, p, jpos[j]);
    }
    if (jown[0] >= 0 && jown[0] == jown[1] && out[20] == out[21] && jpos[1] < jpos[0]) out[22] = 1;
    if (s->mstop) out[22] |= 2;
    out[23] = (uint8_t)s->cur;
    out[24] = s->drawn < 0 ? 0xFF : (uint8_t)s->drawn;
    uint8_t al = 0;
    for (int p = 0; p < s->P; p++) if (s->alive[p]) al |= (uint8_t)(1u << p);
    out[25] = al;
    out[26] = (uint8_t)s->P;
    out[27] = (uint8_t)s->T;
    out[28] = s->winner < 0 ? 0xFF : (uint8_t)s->winner;
}

static void unpack(const uint8_t* in, ost* s) {
    memset(s, 0, sizeof(*s));
    s->P = in[26];
    s->T = in[27];
    for (int t = 0; t < MAXT; t++) s->owner[t] = -1;
    uint32_t rv = rd32(in + 16);
    for (int t = 0; t < s->T; t++) s->rev[t] = (rv >> t) & 1u;
    for (int p = 0; p < s->P; p++) {
        uint32_t m = rd32(in + 4 * p);
        int num[NUMBERED], nn = 0;
        for (int t = 0; t < NUMBERED; t++) if ((m >> t) & 1u) num[nn++] = t;
        int hasj[2] = {(int)((m >> JOKER_BLACK) & 1u), (int)((m >> JOKER_WHITE) & 1u)};
        int white_first = in[22] & 1;
        for (int g = 0; g <= nn; g++) {
            int order[2] = {0, 1};
            if (white_first) { order[0] = 1; order[1] = 0; }
            for (int k = 0; k < 2; k++) {
                int j = order[k];
                if (hasj[j] && in[20 + j] == g) {
                    s->seq[p][s->len[p]++] = JOKER_BLACK + j;
                    s->owner[JOKER_BLACK + j] = p;
                }
            }
            if (g < nn) {
                s->seq[p][s->len[p]++] = num[g];
                s->owner[num[g]] = p;
            }
        }
        s->alive[p] = (in[25] >> p) & 1u;
    }
    s->cur = in[23];
    s->drawn = in[24] == 0xFF ? -1 : in[24];
    s->winner = in[28] == 0xFF ? -1 : in[28];
    s->mstop = (in[22] >> 1) & 1;
}

static int nalive(const ost* s) {
    int n = 0;
    for (int p = 0; p < s->P; p++) n += s->alive[p];
    return n;
}

static int hidden_of(const ost* s, int p) {
    int n = 0;
    for (int i = 0; i < s->len[p]; i++) n += !s->rev[s->seq[p][i]];
    return n;
}

static int revealed_of(const ost* s, int p) { return s->len[p] - hidden_of(s, p); }

/* ------------------------------------------------------------------- rules */

static void put_at(ost* s, int p, int pos, int t) {
    for (int i = s->len[p]; i > pos; i--) s->seq[p][i] = s->seq[p][i - 1];
    s->seq[p][pos] = t;
    s->len[p]++;
    s->owner[t] = p;
}

/* Sorted insertion (Sec. II-A).  A numbered tile goes immediately before the
 * first numbered tile with a larger id (black before white on equal values),
 * so jokers already in that gap stay on its left.  A joker may stand anywhere:
 * its position is uniform over the len+1 insertion points (one word). */
static void insert_tile(ost* s, int p, int t, stream* rng) {
    int pos = s->len[p];
    if (t < NUMBERED) {
        for (int i = 0; i < s->len[p]; i++) {
            int u = s->seq[p][i];
            if (u < NUMBERED && u > t) { pos = i; break; }
        }
    } else {
        pos = pick(next_word(rng), s->len[p] + 1);
    }
    put_at(s, p, pos, t);
}

static int pool_list(const ost* s, int* out) {
    int n = 0;
    for (int t = 0; t < s->T; t++) if (s->owner[t] < 0) out[n++] = t;
    return n;
}

/* Draw phase: a uniform tile of the pool (ascending id order), inserted. */
static void draw_for(ost* s, int p, stream* rng) {
    int pool[MAXT];
    int n = pool_list(s, pool);
    if (n == 0) { s->drawn = -1; return; }
    int t = pool[pick(next_word(rng), n)];
    insert_tile(s, p, t, rng);
    s->drawn = t;
}

/* Every guess the player to move may make, in canonical order: opponents in
 * seat order from cur+1, their face-down slots left to right, then every tile
 * identity that is neither in the guesser's own hand nor face up. */
static int legal_list(const ost* s, int* lq, int* ls, int* lx) {
    int n = 0;
    for (int off = 1; off < s->P; off++) {
        int q = (s->cur + off) % s->P;
        if (!s->alive[q]) continue;
        for (int i = 0; i < s->len[q]; i++) {
            if (s->rev[s->seq[q][i]]) continue;
            for (int x = 0; x < s->T; x++) {
                if (s->owner[x] == s->cur || s->rev[x]) continue;
                lq[n] = q; ls[n] = i; lx[n] = x;
                n++;
            }
        }
    }
    return n;
}

/* The ordering-aware playout policy (not the paper's, a stronger playout
 * for comparison): the same canonical enumeration, keeping for each face-down
 * slot only the identities that fit its place in the sorted row -- a
 * numbered identity must lie strictly between the nearest face-up numbered
 * tiles to the slot's left and right in that row (by tile id, so black
 * before white on equal values); a joker identity fits anywhere.  The slot's
 * own tile always fits, so every face-down slot keeps at least one guess. */
static int legal_list_policy(const ost* s, int policy, int* lq, int* ls, int* lx) {
    if (policy == 0) return legal_list(s, lq, ls, lx);
    int n = 0;
    for (int off = 1; off < s->P; off++) {
        int q = (s->cur + off) % s->P;
        if (!s->alive[q]) continue;
        for (int i = 0; i < s->len[q]; i++) {
            if (s->rev[s->seq[q][i]]) continue;
            int lo = -1, hi = 24;
            for (int j = i - 1; j >= 0; j--) {
                int u = s->seq[q][j];
                if (s->rev[u] && u < 24) { lo = u; break; }
            }
            for (int j = i + 1; j < s->len[q]; j++) {
                int u = s->seq[q][j];
                if (s->rev[u] && u < 24) { hi = u; break; }
            }
            for (int x = 0; x < s->T; x++) {
                if (s->owner[x] == s->cur || s->rev[x]) continue;
                if (x < 24 && !(x > lo && x < hi)) continue;
                lq[n] = q; ls[n] = i; lx[n] = x;
                n++;
            }
        }
    }
    return n;
}

static int guess_is_legal(const ost* s, int q, int slot, int x) {
    if (q == s->cur || q >= s->P || !s->alive[q]) return 0;
    if (slot >= s->len[q] || s->rev[s->seq[q][slot]]) return 0;
    if (x >= s->T || s->owner[x] == s->cur || s->rev[x]) return 0;
    return 1;
}

enum { TURN_OVER = 0, GUESS_AGAIN = 1, GAME_OVER = 2 };

/* Guess resolution (Sec. II-A).  A correct guess turns the target face up;
 * a player with nothing face down is out; the last player standing wins.
 * After a correct guess a playout guesses again iff the next word is below
 * cont_thr; inside the tree the turn always ends (Sec. III-A, simplification
 * 2).  A wrong guess turns the guesser's drawn tile face up, or the leftmost
 * face-down tile when the pool was empty at the draw. */
static int resolve(ost* s, int q, int slot, int x, int in_tree, uint32_t cont_thr, stream* rng) {
    int t = s->seq[q][slot];
    if (t == x) {
        s->rev[t] = 1;
        if (hidden_of(s, q) == 0) s->alive[q] = 0;
        if (nalive(s) == 1) { s->winner = s->cur; return GAME_OVER; }
        if (!in_tree && cont_thr != 0u && next_word(rng) < cont_thr) return GUESS_AGAIN;
        return TURN_OVER;
    }
    int c = s->cur;
    if (s->drawn >= 0) {
        s->rev[s->drawn] = 1;
    } else {
        for (int i = 0; i < s->len[c]; i++) {
            if (!s->rev[s->seq[c][i]]) { s->rev[s->seq[c][i]] = 1; break; }
        }
    }
    if (hidden_of(s, c) == 0) s->alive[c] = 0;
    if (nalive(s) == 1) {
        for (int p = 0; p < s->P; p++) if (s->alive[p]) s->winner = p;
        return GAME_OVER;
    }
    return TURN_OVER;
}

/* The turn passes to the next player still in, who draws. */
static void next_turn(ost* s, stream* rng) {
    int p = s->cur;
    do { p = (p + 1) % s->P; } while (!s->alive[p]);
    s->cur = p;
    draw_for(s, p, rng);
}

/* One action inside the tree (Sec. III-A) or one self-play move: STOP passes
 * the turn; a guess is resolved with no playout coin, and after a correct
 * guess that does not end the game the player keeps the turn (and may stop)
 * when cont is set -- the full game tree of Fig. 2a -- else the turn passes. */
static void tree_step(ost* s, int code, int cont, stream* trng) {
    if (code == STOP) {
        s->mstop = 0;
        next_turn(s, trng);
        return;
    }
    const int q = code >> 10, slot = (code >> 5) & 31, x = code & 31;
    const int correct = s->seq[q][slot] == x;
    if (resolve(s, q, slot, x, 1, 0, NULL) == GAME_OVER) {
        s->mstop = 0;
        return;
    }
    if (correct && cont) {
        s->mstop = 1;
        return;
    }
    s->mstop = 0;
    next_turn(s, trng);
}

static int action_is_legal(const ost* s, int code) {
    if (code == STOP) return s->mstop;
    return guess_is_legal(s, code >> 10, (code >> 5) & 31, code & 31);
}

static _Thread_local int legal_q[MAXLEGAL], legal_s[MAXLEGAL], legal_x[MAXLEGAL];

/* One random playout from a state where the player to move is about to guess
 * (Sec. II-B): uniform guesses among the legal ones until one player is left. */
/* *nsteps (if set) gains the playout's game steps: one per guess, plus one
 * for the continue coin drawn first from a may-stop state. */
static int playout(ost s, uint32_t cont_thr, int policy, stream* rng, uint8_t* trace, int* ntrace, int maxtrace,
                   int64_t* nsteps) {
    if (s.winner >= 0) return s.winner;
    if (s.mstop) {
        /* after a correct guess a playout goes on iff the next word is below cont_thr */
        if (nsteps) ++*nsteps;
        s.mstop = 0;
        if (!(cont_thr != 0u && next_word(rng) < cont_thr)) next_turn(&s, rng);
    }
    for (;;) {
        int n = legal_list_policy(&s, policy, legal_q, legal_s, legal_x);
        int k = pick(next_word(rng), n);
        if (nsteps) ++*nsteps;
        int r = resolve(&s, legal_q[k], legal_s[k], legal_x[k], 0, cont_thr, rng);
        if (r == TURN_OVER) next_turn(&s, rng);
        if (trace && *ntrace < maxtrace) pack(&s, trace + 32 * (*ntrace)++);
        if (r == GAME_OVER) return s.winner;
    }
}

/* -------------------------------------------------------------- root states */

/* Seeded root state (one per index): a deal of cfg->deal tiles to each
 * player in seat order, then a random-policy history of d post-deal draws with
 * d uniform in 0..max_predraw, then the player to move draws.  Histories that
 * end the game or leave some player with more than max_revealed tiles face up
 * are rejected and retried on the same stream; the last attempt uses d = 0. */
#define INIT_ATTEMPTS 16
static void init_one(const or_config* cfg, uint64_t seed, uint32_t index, ost* out) {
    stream rng;
    stream_open(&rng, seed, index, 0, 0, TAG_INIT);
    for (int attempt = 0; attempt < INIT_ATTEMPTS; attempt++) {
        ost s;
        memset(&s, 0, sizeof(s));
        s.P = cfg->nplayers;
        s.T = cfg->ntiles;
        for (int t = 0; t < MAXT; t++) s.owner[t] = -1;
        for (int p = 0; p < s.P; p++) s.alive[p] = 1;
        s.winner = -1;
        for (int p = 0; p < s.P; p++)
            for (int d = 0; d < cfg->deal; d++) draw_for(&s, p, &rng);
        s.drawn = -1;
        s.cur = 0;
        int target = pick(next_word(&rng), cfg->max_predraw + 1);
        int last = attempt == INIT_ATTEMPTS - 1;
        if (last) target = 0;
        int draws = 0, over = 0, pool[MAXT];
        while (draws < target && pool_list(&s, pool) > 0) {
            draw_for(&s, s.cur, &rng);
            draws++;
            for (;;) {
                int n = legal_list(&s, legal_q, legal_s, legal_x);
                int k = pick(next_word(&rng), n);
                int r = resolve(&s, legal_q[k], legal_s[k], legal_x[k], 0, cfg->cont_thr, &rng);
                if (r == GAME_OVER) { over = 1; break; }
                if (r == TURN_OVER) break;
            }
            if (over) break;
            int p = s.cur;
            do { p = (p + 1) % s.P; } while (!s.alive[p]);
            s.cur = p;
        }
        if (over) continue;
        int bad = 0;
        for (int p = 0; p < s.P; p++) bad |= revealed_of(&s, p) > cfg->max_revealed;
        if (bad && !last) continue;
        draw_for(&s, s.cur, &rng);
        *out = s;
        return;
    }
}

int or_init_states(const or_config* cfg, uint64_t seed, int n, uint8_t* out) {
    if (!cfg || n < 0 || cfg->nplayers < 2 || cfg->nplayers > MAXP) return -1;
    if (cfg->ntiles != 24 && cfg->ntiles != 26) return -1;
    if (cfg->deal < 1 || cfg->nplayers * cfg->deal >= cfg->ntiles) return -1;
    for (int i = 0; i < n; i++) {
        ost s;
        init_one(cfg, seed, (uint32_t)i, &s);
        pack(&s, out + 32 * (size_t)i);
    }
    return 0;
}

/* ----------------------------------------------------------- determinizing */

/* Sec. III-A: each simulation draws a set of plausible values for the tiles
 * the observer cannot see.  Reading: uniform over every assignment of the
 * unknown tiles (all tiles minus the observer's hand minus face-up tiles) to
 * the opponents' face-down slots and the pool that is consistent with what
 * the observer sees: each opponent's slot count, the order of numbered tiles
 * (ascending by id), the face-up numbered tiles as anchors, and jokers free to
 * stand in any slot.
 *
 * Counting: the unknown numbered tiles are taken in ascending id order.  For
 * each opponent, the face-down slots between two consecutive face-up numbered
 * anchors form a gap that numbered tiles from that id interval fill in order;
 * slots of a gap left unfilled when the tiles pass its right anchor must hold
 * jokers.  count(i, r, J) is the number of completions when tile u_i is next,
 * r[k] slots of opponent k's current gap are still open, and J unknown jokers
 * are unplaced.  Closing a gap of c slots with r open ones multiplies by
 * C(c, r) * J!/(J-r)! (which slots, which jokers).  Sampling walks the tiles
 * in the same order, choosing the destination (pool first, then opponents
 * from observer+1) in proportion to the completions each leaves, with
 * floor(r64 * total / 2^64) from two words; each close with r > 0 draws one
 * more such index over its C(c, r) * J!/(J-r)! options. */

typedef struct {
    int nq, q[3];
    int nanch[3], anch[3][MAXT];
    int gapsz[3][MAXT + 1];
    int gap_of_slot[3][MAXT]; /* gap index of each face-down slot, -1 for face-up */
    int m, u[NUMBERED];
    int J0, jok[2];
    int G[3][NUMBERED + 1];
    int dim[3];
    uint64_t* memo;
    uint8_t* known;
    size_t stride_i, stride_J;
} detctx;

static uint64_t choose(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; i++) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

static uint64_t joker_close_mult(int c, int r, int J) {
    if (r == 0) return 1;
    if (r > J) return 0;
    uint64_t perm = 1;
    for (int i = 0; i < r; i++) perm *= (uint64_t)(J - i);
    return choose(c, r) * perm;
}

static int det_setup(const ost* s, int obs, detctx* d) {
    memset(d, 0, sizeof(*d));
    d->nq = s->P - 1;
    for (int k = 0; k < d->nq; k++) {
        int q = (obs + 1 + k) % s->P;
        d->q[k] = q;
        int g = 0;
        for (int i = 0; i < s->len[q]; i++) {
            int t = s->seq[q][i];
            if (s->rev[t]) {
                d->gap_of_slot[k][i] = -1;
                if (t < NUMBERED) { d->anch[k][d->nanch[k]++] = t; g++; }
            } else {
                d->gap_of_slot[k][i] = g;
                d->gapsz[k][g]++;
            }
        }
    }
    for (int t = 0; t < s->T; t++) {
        if (s->owner[t] == obs || s->rev[t]) continue;
        if (t < NUMBERED) d->u[d->m++] = t;
        else d->jok[d->J0++] = t;
    }
    for (int k = 0; k < d->nq; k++) {
        for (int i = 0; i < d->m; i++) {
            int g = 0;
            while (g < d->nanch[k] && d->anch[k][g] < d->u[i]) g++;
            d->G[k][i] = g;
        }
        d->G[k][d->m] = d->nanch[k];
        int mx = 0;
        for (int g = 0; g <= d->nanch[k]; g++) if (d->gapsz[k][g] > mx) mx = d->gapsz[k][g];
        d->dim[k] = mx + 1;
    }
    for (int k = d->nq; k < 3; k++) d->dim[k] = 1;
    d->stride_J = (size_t)d->dim[0] * d->dim[1] * d->dim[2];
    d->stride_i = d->stride_J * (size_t)(d->J0 + 1);
    size_t cells = d->stride_i * (size_t)(d->m + 1);
    d->memo = (uint64_t*)calloc(cells, sizeof(uint64_t));
    d->known = (uint8_t*)calloc(cells, 1);
    return d->memo && d->known ? 0 : -1;
}

static void det_free(detctx* d) {
    free(d->memo);
    free(d->known);
}

/* Moving on from layer i (u_i placed or i = -1 at the start) to layer i+1:
 * close every gap the tiles pass.  Returns the multiplier (0 if impossible),
 * and updates r and J.  With rng non-NULL the closes also choose joker slots,
 * recording them in jslot (per opponent, per face-down slot: joker id or -1). */
static uint64_t advance(const detctx* d, int i, int* r, int* J, stream* rng, int jslot[3][MAXT]);

static void place_jokers(const detctx* d, int k, int g, int c, int rr, int* J, int* jleft, stream* rng,
                         int jslot[3][MAXT]) {
    uint64_t opts = joker_close_mult(c, rr, *J);
    if (opts == 0 || rr > 2) return; /* only for a view with no consistent deal */
    uint64_t z = pick64(next_word64(rng), opts);
    uint64_t perms = 1;
    for (int i = 0; i < rr; i++) perms *= (uint64_t)(*J - i);
    uint64_t posidx = z / perms, perm = z % perms;
    int pos[2] = {-1, -1};
    if (rr == 1) {
        pos[0] = (int)posidx;
    } else { /* rr == 2: pairs (a, b), a < b, in lexicographic order */
        uint64_t left = posidx;
        for (int a = 0; a < c && pos[0] < 0; a++) {
            uint64_t cnt = (uint64_t)(c - 1 - a);
            if (left < cnt) { pos[0] = a; pos[1] = a + 1 + (int)left; }
            else left -= cnt;
        }
    }
    int chosen[2];
    if (rr == 1) {
        chosen[0] = jleft[perm];
    } else {
        chosen[0] = jleft[perm == 0 ? 0 : 1];
        chosen[1] = jleft[perm == 0 ? 1 : 0];
    }
    /* map gap-local slot numbers to hand slots */
    int q = d->q[k];
    (void)q;
    for (int e = 0; e < rr; e++) {
        int local = 0;
        for (int i = 0; i < MAXT; i++) {
            if (d->gap_of_slot[k][i] != g) continue;
            if (local == pos[e]) { jslot[k][i] = chosen[e]; break; }
            local++;
        }
    }
    /* remove the chosen jokers from the unplaced list (kept ascending) */
    int nl = 0, keep[2];
    for (int a = 0; a < *J; a++) {
        int used = 0;
        for (int e = 0; e < rr; e++) used |= jleft[a] == chosen[e];
        if (!used) keep[nl++] = jleft[a];
    }
    for (int a = 0; a < nl; a++) jleft[a] = keep[a];
    *J = nl;
}

static _Thread_local int jleft_buf[2];

static uint64_t advance(const detctx* d, int i, int* r, int* J, stream* rng, int jslot[3][MAXT]) {
    uint64_t mult = 1;
    for (int k = 0; k < d->nq; k++) {
        int from = i < 0 ? -1 : d->G[k][i];
        int to = d->G[k][i + 1];
        if (to == from) continue;
        for (int g = from < 0 ? 0 : from; g < to; g++) {
            int open = (g == from) ? r[k] : d->gapsz[k][g];
            uint64_t f = joker_close_mult(d->gapsz[k][g], open, *J);
            if (f == 0) return 0;
            if (rng && open > 0) place_jokers(d, k, g, d->gapsz[k][g], open, J, jleft_buf, rng, jslot);
            else *J -= open;
            mult *= f;
        }
        r[k] = d->gapsz[k][to];
    }
    return mult;
}

static uint64_t finish_mult(const detctx* d, const int* r, int J) {
    uint64_t mult = 1;
    for (int k = 0; k < d->nq; k++) {
        int g = d->nanch[k];
        uint64_t f = joker_close_mult(d->gapsz[k][g], r[k], J);
        if (f == 0) return 0;
        J -= r[k];
        mult *= f;
    }
    return mult;
}

static uint64_t det_count(detctx* d, int i, const int* r, int J) {
    size_t cell = (size_t)i * d->stride_i + (size_t)J * d->stride_J +
                  ((size_t)r[0] * d->dim[1] + (size_t)r[1]) * d->dim[2] + (size_t)r[2];
    if (d->known[cell]) return d->memo[cell];
    uint64_t total = 0;
    if (i == d->m) {
        total = finish_mult(d, r, J);
    } else {
        for (int dest = -1; dest < d->nq; dest++) {
            int r2[3] = {r[0], r[1], r[2]};
            int J2 = J;
            if (dest >= 0) {
                if (r2[dest] == 0) continue;
                r2[dest]--;
            }
            uint64_t f = advance(d, i, r2, &J2, NULL, NULL);
            if (f) total += f * det_count(d, i + 1, r2, J2);
        }
    }
    d->known[cell] = 1;
    d->memo[cell] = total;
    return total;
}

static uint64_t det_total(detctx* d) {
    int r[3] = {0, 0, 0};
    int J = d->J0;
    uint64_t f = advance(d, -1, r, &J, NULL, NULL);
    if (!f) return 0;
    return f * det_count(d, 0, r, J);
}

uint64_t or_det_count(const uint8_t* root, int observer) {
    ost s;
    unpack(root, &s);
    if (observer < 0) observer = s.cur;
    detctx d;
    if (det_setup(&s, observer, &d)) return 0;
    uint64_t n = det_total(&d);
    det_free(&d);
    return n;
}

static int determinize(const ost* root, int obs, stream* rng, ost* out) {
    detctx d;
    if (det_setup(root, obs, &d)) return -1;
    if (det_total(&d) == 0) { det_free(&d); return -2; }
    int jslot[3][MAXT];
    for (int k = 0; k < 3; k++) for (int i = 0; i < MAXT; i++) jslot[k][i] = -1;
    int assigned[3][MAXT], nassigned[3] = {0, 0, 0};
    int r[3] = {0, 0, 0};
    int J = d.J0;
    jleft_buf[0] = d.jok[0];
    jleft_buf[1] = d.jok[1];
    advance(&d, -1, r, &J, rng, jslot);
    for (int i = 0; i < d.m; i++) {
        uint64_t w[4] = {0, 0, 0, 0}, W = 0;
        for (int dest = -1; dest < d.nq; dest++) {
            int r2[3] = {r[0], r[1], r[2]};
            int J2 = J;
            if (dest >= 0) {
                if (r2[dest] == 0) continue;
                r2[dest]--;
            }
            uint64_t f = advance(&d, i, r2, &J2, NULL, NULL);
            if (f) w[dest + 1] = f * det_count(&d, i + 1, r2, J2);
            W += w[dest + 1];
        }
        uint64_t x = pick64(next_word64(rng), W);
        int dest = -1;
        for (int e = 0; e < 4; e++) {
            if (x < w[e]) { dest = e - 1; break; }
            x -= w[e];
        }
        if (dest >= 0) {
            assigned[dest][nassigned[dest]++] = d.u[i];
            r[dest]--;
        }
        advance(&d, i, r, &J, rng, jslot);
    }
    /* the last gaps of each opponent */
    for (int k = 0; k < d.nq; k++) {
        int g = d.nanch[k];
        if (r[k] > 0) place_jokers(&d, k, g, d.gapsz[k][g], r[k], &J, jleft_buf, rng, jslot);
    }
    /* rebuild the opponents' hands */
    *out = *root;
    for (int t = 0; t < out->T; t++)
        if (out->owner[t] >= 0 && out->owner[t] != obs && !out->rev[t]) out->owner[t] = -1;
    for (int k = 0; k < d.nq; k++) {
        int q = d.q[k];
        int next = 0;
        for (int i = 0; i < out->len[q]; i++) {
            if (d.gap_of_slot[k][i] < 0) continue;
            int t = jslot[k][i] >= 0 ? jslot[k][i] : assigned[k][next++];
            out->seq[q][i] = t;
            out->owner[t] = q;
        }
    }
    det_free(&d);
    return 0;
}

int or_determinize(const or_config* cfg, const uint8_t* root, int observer, uint64_t seed, uint32_t tree,
                   uint32_t iter, uint8_t* out) {
    (void)cfg;
    ost s, o;
    unpack(root, &s);
    if (observer < 0) observer = s.cur;
    stream rng;
    stream_open(&rng, seed, tree, 0, iter, TAG_DET);
    int rc = determinize(&s, observer, &rng, &o);
    if (rc) return rc;
    pack(&o, out);
    return 0;
}

/* ----------------------------------------------------------------- rollouts */

/* Per-leaf playouts (Sec. II-B; leaf parallelism): playout j of leaf i of
 * tree t runs on the stream keyed (seed, t) with counter (., j, i, ROLL). */
static int rollout_counted(const or_config* cfg, const uint8_t* leaf, int P, uint64_t seed, uint32_t tree,
                           uint32_t leaf_id, int32_t* wins, int64_t* words, int64_t* steps);

int or_rollout(const or_config* cfg, const uint8_t* leaf, int P, uint64_t seed, uint32_t tree, uint32_t leaf_id,
               int32_t* wins, int64_t* words) {
    return rollout_counted(cfg, leaf, P, seed, tree, leaf_id, wins, words, NULL);
}

/* or_rollout that also adds the playouts' game steps to *steps (if set). */
static int rollout_counted(const or_config* cfg, const uint8_t* leaf, int P, uint64_t seed, uint32_t tree,
                           uint32_t leaf_id, int32_t* wins, int64_t* words, int64_t* steps) {
    ost s;
    unpack(leaf, &s);
    for (int p = 0; p < 4; p++) wins[p] = 0;
    int64_t total = 0;
    if (s.winner >= 0) {
        wins[s.winner] = P;
        if (words) *words = 0;
        return 0;
    }
    for (int j = 0; j < P; j++) {
        stream rng;
        stream_open(&rng, seed, tree, (uint32_t)j, leaf_id, TAG_ROLL);
        int w = playout(s, cfg->cont_thr, cfg->policy, &rng, NULL, NULL, 0, steps);
        wins[w]++;
        total += rng.words;
    }
    if (words) *words = total;
    return 0;
}

int or_playout_trace(const or_config* cfg, const uint8_t* leaf, uint64_t seed, uint32_t tree, uint32_t j,
                     uint32_t leaf_id, uint8_t* trace, int maxtrace) {
    ost s;
    unpack(leaf, &s);
    stream rng;
    stream_open(&rng, seed, tree, j, leaf_id, TAG_ROLL);
    int n = 0;
    playout(s, cfg->cont_thr, cfg->policy, &rng, trace, &n, maxtrace, NULL);
    return n;
}

int or_legal_count(const uint8_t* state) {
    ost s;
    unpack(state, &s);
    return legal_list(&s, legal_q, legal_s, legal_x);
}

/* One move of a game played out by search agents (the workload's self-play
 * games), under the game model the trees search: the seat to move makes the
 * guess `code` (seat << 10 | slot << 5 | identity) on the true state, or STOP
 * when it may; with cont = 0 the turn ends after any guess (Sec. III-A,
 * simplification 2), with cont = 1 a correct guess keeps the turn (Fig. 2a);
 * when the turn passes the next seat still in draws on the stream (seed,
 * game, turn, tag 5).  Returns 0; 1 if the game was already over; -1 if the
 * action is not legal (the state is copied unchanged). */
int or_play_move(const uint8_t* in, int code, int cont, uint64_t seed, uint32_t game, uint32_t turn, uint8_t* out) {
    ost s;
    unpack(in, &s);
    if (s.winner >= 0) {
        pack(&s, out);
        return 1;
    }
    if (code < 0 || !action_is_legal(&s, code)) {
        pack(&s, out);
        return -1;
    }
    stream rng;
    stream_open(&rng, seed, game, 0, turn, TAG_PLAY);
    tree_step(&s, code, cont, &rng);
    pack(&s, out);
    return 0;
}

/* The legal guesses of a state in canonical order (opponents from the mover
 * + 1, slots left to right, identities ascending) as action codes, all of
 * them (policy 0) or those the ordering-aware playout policy keeps (policy
 * 1); returns their number (at most 3 * 26 * 26). */
int or_legal_actions(const uint8_t* state, int policy, int32_t* codes) {
    ost s;
    unpack(state, &s);
    const int n = legal_list_policy(&s, policy, legal_q, legal_s, legal_x);
    for (int a = 0; a < n; a++) codes[a] = (legal_q[a] << 10) | (legal_s[a] << 5) | legal_x[a];
    return n;
}

/* --------------------------------------------------------------------- UCT */

/* Natural log in IEEE single precision: x = m * 2^e with m in
 * [sqrt(1/2), sqrt(2)); ln x = e ln 2 + 2 atanh(z), z = (m-1)/(m+1), the
 * series z + z^3/3 + ... + z^11/11 (|z| <= 0.1716, so the next term is below
 * 2^-30 of the sum) evaluated by Horner from the 11th power down.  Plain
 * float operations in a fixed order; ln 2 is the float nearest to it. */
float or_lnf(float x) {
    union { float f; uint32_t u; } v;
    v.f = x;
    int e = (int)((v.u >> 23) & 0xFF) - 127;
    v.u = (v.u & 0x007FFFFFu) | 0x3F800000u;
    float m = v.f;
    if (m > 1.41421354f) {
        m = m * 0.5f;
        e = e + 1;
    }
    float z = (m - 1.0f) / (m + 1.0f);
    float z2 = z * z;
    float p = 1.0f / 11.0f;
    for (int k = 4; k >= 0; k--) p = p * z2 + 1.0f / (float)(2 * k + 1);
    float lnm = 2.0f * (z * p);
    return (float)e * 0.693147182f + lnm;
}

/* Score of a child (UCB1 with visits counted in playouts), in IEEE single
 * precision:
 *   mean = wins / n;  explore = (c * sqrt(ln N)) * (1 / sqrt(n));  score = mean + explore
 * with N the parent's visits, evaluated in exactly this order. */
static float uct_score(float c_sqrt_lnN, int32_t w, int32_t n) {
    float mean = (float)w / (float)n;
    float rs = 1.0f / sqrtf((float)n);
    return mean + c_sqrt_lnN * rs;
}

static int canon_rank(int code, int cur, int P) {
    if (code == STOP) return 0;
    int q = code >> 10;
    return 1 + (((((q - cur - 1) % P + P) % P) << 10) | (code & 1023));
}

typedef struct {
    int n, cap;
    int32_t *action, *parent, *visits, *wins, *child, *sib, *last;
    uint64_t* key; /* SET nodes: the assignment they stand for (set_key) */
} otree;

/* The plausible-number set of a determinization seen by observer obs: every
 * other seat's hand (bitmask), then the joker gaps and the white-first flag,
 * in two words. */
static void set_key(const ost* s, int obs, uint64_t key[2]) {
    uint8_t b[32];
    pack(s, b);
    uint64_t h[3] = {0, 0, 0};
    int k = 0;
    for (int p = 0; p < s->P; p++)
        if (p != obs) h[k++] = rd32(b + 4 * p);
    key[0] = h[0] | (h[1] << 32);
    key[1] = h[2] | ((uint64_t)b[20] << 32) | ((uint64_t)b[21] << 40) | ((uint64_t)(b[22] & 1u) << 48);
}

static int tree_new_node(otree* t, int parent, int code) {
    int id = t->n++;
    t->action[id] = code;
    t->parent[id] = parent;
    t->visits[id] = 0;
    t->wins[id] = 0;
    t->child[id] = -1;
    t->sib[id] = -1;
    t->last[id] = -1;
    if (parent >= 0) {
        if (t->child[parent] < 0) t->child[parent] = id;
        else t->sib[t->last[parent]] = id;
        t->last[parent] = id;
    }
    return id;
}

int or_value_forward(const float* prm, const uint8_t* packed, double* probs);

/* One search of `budget` iterations from `root` (observer = player to move):
 * determinize, descend by UCT among children legal in this determinization,
 * expand the first legal action without a child (canonical order) while the
 * depth is below d_max, score the leaf, and add the playout count to every
 * visit and the leaf's credit for each node's mover to its wins (a node's
 * wins are those of the seat that moved into it; the root's are the
 * observer's).  The leaf's credit per seat: a leaf that ended inside the tree
 * gives all `playouts` to its winner; otherwise, with value_prm NULL, the
 * wins of `playouts` random playouts (Sec. II-B); with value_prm set (value
 * mode, no counterpart in the paper: the learned evaluator stands in for the
 * playouts), round(p_s * playouts) = floor(p_s * playouts + 0.5) for each
 * seat s, p the network's win probabilities of the leaf. */
static int mcts_run(const or_config* cfg, const uint8_t* root_packed, uint64_t seed, uint32_t tree_id, int budget,
                    const float* value_prm, int32_t* nodes_out, int* n_nodes_out, int32_t* best_out, int64_t* work) {
    ost root;
    unpack(root_packed, &root);
    int obs = root.cur;
    int P = cfg->playouts;
    otree t;
    t.cap = budget + 1;
    t.n = 0;
    int32_t* mem = (int32_t*)malloc(sizeof(int32_t) * 7 * (size_t)t.cap);
    t.key = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (size_t)t.cap);
    if (!mem || !t.key) { free(mem); free(t.key); return -1; }
    t.action = mem; t.parent = mem + t.cap; t.visits = mem + 2 * t.cap; t.wins = mem + 3 * t.cap;
    t.child = mem + 4 * t.cap; t.sib = mem + 5 * t.cap; t.last = mem + 6 * t.cap;
    tree_new_node(&t, -1, 0);
    int rc = 0;
    for (int it = 0; it < budget && rc == 0; it++) {
        ost s;
        stream drng, trng;
        stream_open(&drng, seed, tree_id, 0, (uint32_t)it, TAG_DET);
        stream_open(&trng, seed, tree_id, 0, (uint32_t)it, TAG_TREE);
        if (determinize(&root, obs, &drng, &s)) { rc = -2; break; }
        int path[64], mover[64], np = 0;
        path[np] = 0;
        mover[np++] = obs;
        int node = 0, depth = 0;
        if (cfg->vanilla) {
            /* the root's child for this determinization's plausible set, or
             * a new one (this iteration's expansion; its leaf is the root
             * determinized) */
            uint64_t key[2];
            set_key(&s, obs, key);
            int c = t.child[0];
            while (c >= 0 && !(t.key[2 * c] == key[0] && t.key[2 * c + 1] == key[1])) c = t.sib[c];
            int fresh = c < 0;
            if (fresh) {
                c = tree_new_node(&t, 0, SET);
                t.key[2 * c] = key[0];
                t.key[2 * c + 1] = key[1];
            }
            path[np] = c;
            mover[np++] = obs;
            node = c;
            if (fresh) depth = cfg->d_max; /* no descent below a node created in this iteration */
        }
        while (s.winner < 0 && depth < cfg->d_max) {
            /* the node's actions in canonical order: STOP when the mover may stop, then the legal guesses */
            int n = legal_list(&s, legal_q, legal_s, legal_x);
            int fresh_code = -1;
            for (int a = s.mstop ? -1 : 0; a < n && fresh_code < 0; a++) {
                int code = a < 0 ? STOP : (legal_q[a] << 10) | (legal_s[a] << 5) | legal_x[a];
                int found = 0;
                for (int c = t.child[node]; c >= 0; c = t.sib[c]) found |= t.action[c] == code;
                if (!found) fresh_code = code;
            }
            int who = s.cur;
            if (fresh_code >= 0) {
                int c = tree_new_node(&t, node, fresh_code);
                tree_step(&s, fresh_code, cfg->tree_continue, &trng);
                path[np] = c;
                mover[np++] = who;
                break;
            }
            float lnN = or_lnf((float)t.visits[node]);
            float csl = (float)cfg->c_uct * sqrtf(lnN);
            int best = -1, best_rank = 0;
            float best_score = 0.0f;
            for (int c = t.child[node]; c >= 0; c = t.sib[c]) {
                int code = t.action[c];
                if (!action_is_legal(&s, code)) continue;
                float sc = uct_score(csl, t.wins[c], t.visits[c]);
                int rank = canon_rank(code, s.cur, s.P);
                if (best < 0 || sc > best_score || (sc == best_score && rank < best_rank)) {
                    best = c; best_score = sc; best_rank = rank;
                }
            }
            tree_step(&s, t.action[best], cfg->tree_continue, &trng);
            path[np] = best;
            mover[np++] = who;
            node = best;
            depth++;
        }
        int32_t wins[4] = {0, 0, 0, 0};
        if (s.winner >= 0) {
            wins[s.winner] = P;
        } else if (value_prm) {
            uint8_t leaf[32];
            double p[4];
            pack(&s, leaf);
            if (or_value_forward(value_prm, leaf, p)) { rc = -1; break; }
            for (int q = 0; q < 4; q++) wins[q] = (int32_t)floor(p[q] * (double)P + 0.5);
        } else {
            uint8_t leaf[32];
            pack(&s, leaf);
            int64_t nw = 0;
            rollout_counted(cfg, leaf, P, seed, tree_id, (uint32_t)it, wins, &nw, work ? work + 1 : NULL);
            if (work) work[0] += nw;
        }
        for (int k = 0; k < np; k++) {
            t.visits[path[k]] += P;
            t.wins[path[k]] += wins[mover[k]];
        }
    }
    if (rc == 0) {
        if (nodes_out) {
            for (int i = 0; i < t.n; i++) {
                nodes_out[4 * i + 0] = t.action[i];
                nodes_out[4 * i + 1] = t.parent[i];
                nodes_out[4 * i + 2] = t.visits[i];
                nodes_out[4 * i + 3] = t.wins[i];
            }
        }
        if (n_nodes_out) *n_nodes_out = t.n;
        if (best_out && !cfg->vanilla) {
            /* decision: most visits, ties to the lowest canonical rank */
            int best = -1;
            for (int c = t.child[0]; c >= 0; c = t.sib[c]) {
                if (best < 0 || t.visits[c] > t.visits[best] ||
                    (t.visits[c] == t.visits[best] &&
                     canon_rank(t.action[c], obs, root.P) < canon_rank(t.action[best], obs, root.P)))
                    best = c;
            }
            best_out[0] = best < 0 ? -1 : t.action[best];
            best_out[1] = best < 0 ? 0 : t.visits[best];
            best_out[2] = best < 0 ? 0 : t.wins[best];
            best_out[3] = t.visits[0];
        } else if (best_out) {
            /* vanilla: an action's visits and wins summed over every plausible set */
            static _Thread_local int32_t av[4096], aw[4096];
            memset(av, 0, sizeof(av));
            memset(aw, 0, sizeof(aw));
            for (int c = t.child[0]; c >= 0; c = t.sib[c])
                for (int g = t.child[c]; g >= 0; g = t.sib[g]) {
                    av[t.action[g]] += t.visits[g];
                    aw[t.action[g]] += t.wins[g];
                }
            int best = -1;
            for (int a = 0; a < 4096; a++) {
                if (av[a] == 0) continue;
                if (best < 0 || av[a] > av[best] ||
                    (av[a] == av[best] && canon_rank(a, obs, root.P) < canon_rank(best, obs, root.P)))
                    best = a;
            }
            best_out[0] = best;
            best_out[1] = best < 0 ? 0 : av[best];
            best_out[2] = best < 0 ? 0 : aw[best];
            best_out[3] = t.visits[0];
        }
    }
    free(mem);
    free(t.key);
    return rc;
}

int or_mcts(const or_config* cfg, const uint8_t* root_packed, uint64_t seed, uint32_t tree_id, int budget,
            int32_t* nodes_out, int* n_nodes_out, int32_t* best_out) {
    return mcts_run(cfg, root_packed, seed, tree_id, budget, NULL, nodes_out, n_nodes_out, best_out, NULL);
}

/* The search's playout work: work[0] random words, work[1] game steps (one
 * per guess, plus one per continue coin drawn first from a may-stop leaf). */
int or_mcts_work(const or_config* cfg, const uint8_t* root_packed, uint64_t seed, uint32_t tree_id, int budget,
                 int64_t* work) {
    work[0] = work[1] = 0;
    return mcts_run(cfg, root_packed, seed, tree_id, budget, NULL, NULL, NULL, NULL, work);
}

/* The same search in value mode: every fresh leaf that did not end inside the
 * tree is credited from the value network (parameters `prm`, layout below)
 * instead of playouts. */
int or_mcts_value(const or_config* cfg, const uint8_t* root_packed, uint64_t seed, uint32_t tree_id, int budget,
                  const float* prm, int32_t* nodes_out, int* n_nodes_out, int32_t* best_out) {
    if (!prm) return -1;
    return mcts_run(cfg, root_packed, seed, tree_id, budget, prm, nodes_out, n_nodes_out, best_out, NULL);
}

/* ------------------------------------------------------------- value net */

/* Leaf evaluator of the workload (no counterpart in the paper's method; the
 * method's own leaf evaluation is the random playout).  Input features of a
 * state, from the seat to move (cur), seats relative to cur:
 *   [0, 182)   per tile t < 26: owner one-hot over 4 relative seats, then
 *              face-down / face-up (2), then drawn this turn (1) -- 7 each;
 *              zeros for tiles in the pool or absent from the game;
 *   [182, 611) per opponent k = 1..3 (relative), per slot s < 11 of its row:
 *              13 values (12 numbers + joker): a face-up slot marks its own
 *              value; a face-down slot marks every value v for which some tile
 *              unknown to the mover (not in its hand, not face up) of value v
 *              fits between the slot's face-up numbered neighbours, plus the
 *              joker if an unknown joker exists;
 *   [611, 640) zero padding.
 * Network: 640 -> 512 -> 512 -> 512 (GELU, tanh form) -> 4 logits over
 * relative seats; softmax over the seats in play; output per absolute seat.
 * Parameter layout (floats): W1[512][640], b1[512], W2[512][512], b2[512],
 * W3[512][512], b3[512], W4[4][512], b4[4].  Computed in double. */
#define VF 640
#define VH 512
#define VP (VH * VF + VH + VH * VH + VH + VH * VH + VH + 4 * VH + 4)

int or_value_nparams(void) { return VP; }

int or_value_features(const uint8_t* packed, float* out) {
    ost s;
    unpack(packed, &s);
    for (int i = 0; i < VF; i++) out[i] = 0.0f;
    int c = s.cur, P = s.P;
    for (int t = 0; t < s.T; t++) {
        if (s.owner[t] < 0) continue;
        int rel = ((s.owner[t] - c) % P + P) % P;
        out[7 * t + rel] = 1.0f;
        out[7 * t + 4 + (s.rev[t] ? 1 : 0)] = 1.0f;
        if (t == s.drawn) out[7 * t + 6] = 1.0f;
    }
    int unknown[MAXT];
    for (int t = 0; t < MAXT; t++) unknown[t] = t < s.T && s.owner[t] != c && !s.rev[t];
    for (int k = 1; k < 4; k++) {
        if (k >= P) break;
        int q = (c + k) % P;
        for (int i = 0; i < s.len[q] && i < 11; i++) {
            float* f = out + 182 + ((k - 1) * 11 + i) * 13;
            int t = s.seq[q][i];
            if (s.rev[t]) {
                f[t < NUMBERED ? t / 2 : 12] = 1.0f;
                continue;
            }
            int lo = -1, hi = NUMBERED; /* face-up numbered neighbours */
            for (int j = i - 1; j >= 0; j--) {
                int u = s.seq[q][j];
                if (s.rev[u] && u < NUMBERED) { lo = u; break; }
            }
            for (int j = i + 1; j < s.len[q]; j++) {
                int u = s.seq[q][j];
                if (s.rev[u] && u < NUMBERED) { hi = u; break; }
            }
            for (int u = 0; u < NUMBERED; u++)
                if (unknown[u] && u > lo && u < hi) f[u / 2] = 1.0f;
            if (unknown[JOKER_BLACK] || unknown[JOKER_WHITE]) f[12] = 1.0f;
        }
    }
    return 0;
}

/* GELU in its tanh form (Hendrycks and Gimpel, 2016):
 * 0.5 x (1 + tanh(u)), u = sqrt(2/pi) (x + 0.044715 x^3), and its derivative
 * 0.5 (1 + t) + 0.5 x (1 - t^2) sqrt(2/pi) (1 + 3 * 0.044715 x^2), t = tanh(u). */
static double gelu_d(double x) {
    const double k = sqrt(2.0 / 3.14159265358979323846);
    return 0.5 * x * (1.0 + tanh(k * (x + 0.044715 * x * x * x)));
}
static double gelu_grad_d(double x) {
    const double k = sqrt(2.0 / 3.14159265358979323846);
    const double t = tanh(k * (x + 0.044715 * x * x * x));
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * k * (1.0 + 3.0 * 0.044715 * x * x);
}

typedef struct {
    double x[VF], z1[VH], h1[VH], z2[VH], h2[VH], z3[VH], h3[VH], z4[4], p[4];
    int P, cur;
} vfwd;

static void dense(const float* W, const float* b, const double* in, int nin, int nout, double* out) {
    for (int o = 0; o < nout; o++) {
        double acc = b[o];
        for (int i = 0; i < nin; i++) acc += (double)W[(size_t)o * nin + i] * in[i];
        out[o] = acc;
    }
}

static void value_forward(const float* prm, const uint8_t* packed, vfwd* f) {
    float xf[VF];
    or_value_features(packed, xf);
    for (int i = 0; i < VF; i++) f->x[i] = xf[i];
    const float* W1 = prm;
    const float* b1 = W1 + VH * VF;
    const float* W2 = b1 + VH;
    const float* b2 = W2 + VH * VH;
    const float* W3 = b2 + VH;
    const float* b3 = W3 + VH * VH;
    const float* W4 = b3 + VH;
    const float* b4 = W4 + 4 * VH;
    dense(W1, b1, f->x, VF, VH, f->z1);
    for (int i = 0; i < VH; i++) f->h1[i] = gelu_d(f->z1[i]);
    dense(W2, b2, f->h1, VH, VH, f->z2);
    for (int i = 0; i < VH; i++) f->h2[i] = gelu_d(f->z2[i]);
    dense(W3, b3, f->h2, VH, VH, f->z3);
    for (int i = 0; i < VH; i++) f->h3[i] = gelu_d(f->z3[i]);
    dense(W4, b4, f->h3, VH, 4, f->z4);
    f->P = packed[26];
    f->cur = packed[23];
    double mx = -1e300, sum = 0.0;
    for (int r = 0; r < f->P; r++) if (f->z4[r] > mx) mx = f->z4[r];
    for (int r = 0; r < 4; r++) f->p[r] = r < f->P ? exp(f->z4[r] - mx) : 0.0;
    for (int r = 0; r < f->P; r++) sum += f->p[r];
    for (int r = 0; r < f->P; r++) f->p[r] /= sum;
}

/* Win probability per absolute seat. */
int or_value_forward(const float* prm, const uint8_t* packed, double* probs) {
    vfwd* f = (vfwd*)malloc(sizeof(vfwd));
    if (!f) return -1;
    value_forward(prm, packed, f);
    for (int s = 0; s < 4; s++) probs[s] = 0.0;
    for (int r = 0; r < f->P; r++) probs[(f->cur + r) % f->P] = f->p[r];
    free(f);
    return 0;
}

/* Mean cross-entropy over n states against soft labels (4 per state, by
 * absolute seat) and its gradient with respect to every parameter. */
double or_value_loss_grad(const float* prm, const uint8_t* states, const float* labels, int n, double* grad) {
    for (int i = 0; i < VP; i++) grad[i] = 0.0;
    const float* W2 = prm + VH * VF + VH;
    const float* W3 = W2 + VH * VH + VH;
    const float* W4 = W3 + VH * VH + VH;
    double* gW1 = grad;
    double* gb1 = gW1 + VH * VF;
    double* gW2 = gb1 + VH;
    double* gb2 = gW2 + VH * VH;
    double* gW3 = gb2 + VH;
    double* gb3 = gW3 + VH * VH;
    double* gW4 = gb3 + VH;
    double* gb4 = gW4 + 4 * VH;
    vfwd* f = (vfwd*)malloc(sizeof(vfwd));
    double* d = (double*)malloc(sizeof(double) * 3 * VH);
    if (!f || !d) { free(f); free(d); return -1.0; }
    double* dh = d;
    double* dz = d + VH;
    double* dtmp = d + 2 * VH;
    double loss = 0.0;
    for (int b = 0; b < n; b++) {
        value_forward(prm, states + 32 * (size_t)b, f);
        double dz4[4] = {0, 0, 0, 0};
        for (int r = 0; r < f->P; r++) {
            double y = labels[4 * b + (f->cur + r) % f->P];
            if (y > 0) loss -= y * log(f->p[r]);
            dz4[r] = (f->p[r] - y) / n;
        }
        for (int r = 0; r < 4; r++) {
            gb4[r] += dz4[r];
            for (int i = 0; i < VH; i++) gW4[r * VH + i] += dz4[r] * f->h3[i];
        }
        for (int i = 0; i < VH; i++) {
            double acc = 0.0;
            for (int r = 0; r < 4; r++) acc += dz4[r] * W4[r * VH + i];
            dz[i] = acc * gelu_grad_d(f->z3[i]);
        }
        for (int o = 0; o < VH; o++) {
            gb3[o] += dz[o];
            for (int i = 0; i < VH; i++) gW3[(size_t)o * VH + i] += dz[o] * f->h2[i];
        }
        for (int i = 0; i < VH; i++) {
            double acc = 0.0;
            for (int o = 0; o < VH; o++) acc += dz[o] * W3[(size_t)o * VH + i];
            dh[i] = acc;
        }
        for (int i = 0; i < VH; i++) dtmp[i] = dh[i] * gelu_grad_d(f->z2[i]);
        for (int o = 0; o < VH; o++) {
            gb2[o] += dtmp[o];
            for (int i = 0; i < VH; i++) gW2[(size_t)o * VH + i] += dtmp[o] * f->h1[i];
        }
        for (int i = 0; i < VH; i++) {
            double acc = 0.0;
            for (int o = 0; o < VH; o++) acc += dtmp[o] * W2[(size_t)o * VH + i];
            dh[i] = acc;
        }
        for (int i = 0; i < VH; i++) dz[i] = dh[i] * gelu_grad_d(f->z1[i]);
        for (int o = 0; o < VH; o++) {
            gb1[o] += dz[o];
            for (int i = 0; i < VF; i++) gW1[(size_t)o * VF + i] += dz[o] * f->x[i];
        }
    }
    free(f);
    free(d);
    return loss / n;
}

/* One AdamW step (Loshchilov and Hutter, "Decoupled Weight Decay
 * Regularization", ICLR 2019; Adam of Kingma and Ba, ICLR 2015), in double,
 * over the value network's parameters in the layout above:
 *   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
 *   mhat = m / (1 - b1^t);  vhat = v / (1 - b2^t);
 *   w <- w - lr (mhat / (sqrt(vhat) + eps) + wd w)
 * with t the step number after this update (1 for the first) and the weight
 * decay applied to the weight matrices only, not to the biases. */
int or_adamw_step(double* w, double* m, double* v, const double* g, long long t, double lr, double b1, double b2,
                  double eps, double wd) {
    if (t < 1) return -1;
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    const long long b1o = (long long)VH * VF, b2o = b1o + VH + (long long)VH * VH, b3o = b2o + VH + (long long)VH * VH,
                    b4o = b3o + VH + 4LL * VH;
    for (long long i = 0; i < VP; i++) {
        const int is_bias = (i >= b1o && i < b1o + VH) || (i >= b2o && i < b2o + VH) || (i >= b3o && i < b3o + VH) ||
                            i >= b4o;
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        const double mhat = m[i] / c1, vhat = v[i] / c2;
        double upd = mhat / (sqrt(vhat) + eps);
        if (!is_bias) upd += wd * w[i];
        w[i] -= lr * upd;
    }
    return 0;
}

/* Root-parallel merge (Sec. III-B): the decision of K searches of one root,
 * given their node tables (rows [action, parent, visits, wins] in creation
 * order, row 0 the root), concatenated, counts[k] rows each.  Each action's
 * root-child visits and wins are summed over the K tables (vanilla: the
 * children of every plausible-set node, the root's children there); the
 * decision is the action with most visits, ties to the lowest canonical rank.
 * out[4]: action (-1 if none), its visits, its wins, the summed root visits. */
int or_root_merge(const uint8_t* root_packed, int K, const int32_t* tables, const int32_t* counts, int vanilla,
                  int32_t* out) {
    ost root;
    unpack(root_packed, &root);
    static _Thread_local int32_t av[4096], aw[4096];
    memset(av, 0, sizeof(av));
    memset(aw, 0, sizeof(aw));
    int32_t root_visits = 0;
    const int32_t* t = tables;
    for (int k = 0; k < K; k++) {
        const int n = counts[k];
        if (n < 1) return -1;
        root_visits += t[2];
        for (int i = 1; i < n; i++) {
            const int32_t action = t[4 * i], parent = t[4 * i + 1];
            const int counted = vanilla ? (parent > 0 && t[4 * parent + 1] == 0) : parent == 0;
            if (!counted) continue;
            if (action < 0 || action >= 4096) return -1;
            av[action] += t[4 * i + 2];
            aw[action] += t[4 * i + 3];
        }
        t += 4 * n;
    }
    int best = -1;
    for (int a = 0; a < 4096; a++) {
        if (av[a] == 0) continue;
        if (best < 0 || av[a] > av[best] ||
            (av[a] == av[best] && canon_rank(a, root.cur, root.P) < canon_rank(best, root.cur, root.P)))
            best = a;
    }
    out[0] = best;
    out[1] = best < 0 ? 0 : av[best];
    out[2] = best < 0 ? 0 : aw[best];
    out[3] = root_visits;
    return 0;
}
