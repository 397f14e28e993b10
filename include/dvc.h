/*
 * dvc.h -- C ABI of libdvc, a GB300 (sm_103a) engine for the Da Vinci Code
 * Monte Carlo Tree Search of arXiv 2403.10720.
 *
 * What it computes (paper sections):
 *   Sec. II-A   the game: 24 numbered tiles (values 0-11, black and white) plus
 *               two jokers in the 26-tile variant; each player holds a hidden
 *               row kept in ascending order; a turn is a draw with sorted
 *               insertion, then guesses at opponents' face-down tiles; a
 *               correct guess turns the tile face up and allows another
 *               guess, a wrong one turns the guesser's drawn tile face up and
 *               ends the turn; the last player with face-down tiles wins.
 *   Sec. II-B   MCTS: select, expand, simulate by random playout, backpropagate.
 *   Sec. III-A  the simplified tree: a node is a guess (slot, identity); the
 *               unseen tiles are re-sampled per simulation (determinization);
 *               inside the tree a correct guess ends the turn; expansion stops
 *               at a fixed depth.
 *   Sec. III-B  many searches run in parallel and their root statistics merge.
 *
 * Conventions, for every entry point:
 *   - returns 0 on success or a negative DVC_E_* code; dvc_last_error() gives
 *     a message.  No C++ exception crosses this boundary.
 *   - pointers named d_* are DEVICE memory owned by the caller (for example
 *     PyTorch tensors passed as raw pointers), of the context's device (or
 *     managed memory): a pointer into another GPU's memory is DVC_E_INVALID;
 *     h_* are host memory owned by the caller.  The library owns only its
 *     context, forests and workspace.
 *   - work is enqueued on the given CUDA stream (cudaStream_t passed as void*;
 *     NULL = legacy default stream); outputs are valid after that stream is
 *     synchronised.  Arguments are validated on the host before anything is
 *     enqueued: a call that returns an error has enqueued nothing.
 *   - errors found by a kernel (a determinization table larger than its
 *     capacity, a node arena exhausted) are latched in a device flag of the
 *     context; dvc_check() synchronises the device and reports them.
 *   - a context is bound to the device given at creation; calls that enqueue
 *     work make that device current on the calling thread.
 *   - calls on one context or forest from several host threads at once are
 *     not supported.
 *
 * Random numbers: Philox-4x32-10 (Salmon et al., SC'11).  A stream is keyed
 * (low 32 bits of seed, tree id) with counter (block, playout j, iteration or
 * leaf i, tag + 16 * high 32 bits of seed), tag 1 = root-state generation,
 * 2 = determinization, 3 = draws inside the tree, 4 = playouts, 5 = draws of
 * self-play games (dvc_play_move).  Words of a
 * block are consumed in order.  Every result is therefore a pure function of
 * (seed, tree id, iteration, playout index) and does not depend on the thread
 * mapping, the launch shape or the order in which playouts finish.
 */
#ifndef DVC_H
#define DVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DVC_OK 0
#define DVC_E_INVALID (-1)     /* bad argument: size, null pointer, host pointer where device is needed */
#define DVC_E_OOM (-2)         /* device allocation failed, or a forest arena is full */
#define DVC_E_CUDA (-3)        /* a CUDA runtime call failed */
#define DVC_E_TIMEOUT (-4)     /* a bounded device wait gave up */
#define DVC_E_UNSUPPORTED (-5) /* a size beyond a documented capacity */
#define DVC_E_INTERNAL (-6)    /* a device-side invariant failed: a playout still running after 128 guesses
                                  (a game has at most |T| guesses, each turning one tile face up); that
                                  playout credits nobody */

#define DVC_MODE_ROLLOUT 0 /* leaves are scored by random playouts (Sec. II-B) */
#define DVC_MODE_VALUE 1   /* leaves are scored by the value network */

/*
 * One game position, 32 bytes, identical on host and device.
 * Tile ids: numbered tile t = 2*value + colour (colour 0 black, 1 white),
 * 0..23; jokers 24 (black) and 25 (white).  A hand is the set of tiles a
 * player holds; its left-to-right order is derived: numbered tiles ascend by
 * id (black before white on equal values), each joker stands after joker_gap
 * numbered tiles, and two jokers of one hand with the same gap are ordered
 * black first unless bit 0 of flags is set.  Bit 1 of flags marks a seat
 * to move that has guessed correctly this turn and may stop (the full game
 * tree, dvc_config.tree_continue).  The pool is every tile of the game held
 * by nobody.
 */
typedef struct dvc_state {
    uint32_t hand[4];     /* tile bitmask per seat (unused seats 0) */
    uint32_t revealed;    /* face-up tiles */
    uint8_t joker_gap[2]; /* numbered tiles left of joker 24 / 25 in its owner's hand; 0 in the pool */
    uint8_t flags;        /* bit 0: jokers share owner and gap, white first; bit 1: may stop (see above) */
    uint8_t cur;          /* seat to move; it has drawn and is about to guess */
    uint8_t drawn;        /* tile drawn this turn, 0xFF if the pool was empty */
    uint8_t alive;        /* bitmask of seats with a face-down tile */
    uint8_t nplayers;     /* 2..4 */
    uint8_t ntiles;       /* 24 or 26 */
    uint8_t winner;       /* 0xFF while the game runs */
    uint8_t pad[3];       /* zero */
} dvc_state;

/*
 * Game and search parameters.  Readings of what the paper leaves open:
 * cont_thr -- after a correct guess a playout guesses again iff the next
 * random word is below cont_thr (2^31 = probability 1/2; 0 = never, and no
 * word is drawn); inside the tree the turn always ends (Sec. III-A).
 * d_max -- the expansion depth limit of Sec. III-A, in guess plies below the
 * root.  c_uct -- the UCB1 exploration constant.  policy -- the playout guess
 * rule: 0 = uniform over the legal guesses (Sec. II-B, the paper's random
 * playout); 1 = ordering-aware, not the paper's: for each face-down slot only
 * the identities that fit between its nearest face-up numbered neighbours in
 * the sorted row (jokers anywhere), uniform over the kept (slot, identity)
 * pairs in the same canonical order, one word per guess.  It changes
 * playouts only; the tree's actions stay the legal guesses.
 * tree_continue -- 0: inside the tree a correct guess ends the turn (Sec.
 * III-A, simplification 2); 1: the full game tree of Fig. 2a: after a correct
 * guess that does not end the game the player keeps the turn, and its node
 * offers STOP (action code 0xFFF, first in canonical order) beside the legal
 * guesses; STOP passes the turn.  The same rule governs dvc_play_move.
 * vanilla -- 0: the paper's MCTS-dvc tree, whose root's children are the
 * guesses (Sec. III-A); 1: vanilla MCTS-dvc, the baseline Sec. III-A sets it
 * against: the root's children are plausible-number sets (action code 0xFFE),
 * one per distinct assignment of the tiles the observer cannot see (every
 * other seat's hand with its jokers' places); each iteration enters the set
 * of its determinization, and a set not seen before is that iteration's
 * expansion, scored from the determinized root.  Below a set the tree is the
 * usual guess tree (d_max counts plies below the set).  The decision sums
 * each action's visits and wins over all sets (dvc_root_stats).  Forests
 * only: dvc_server_create returns DVC_E_UNSUPPORTED.
 */
typedef struct dvc_config {
    int32_t nplayers;         /* 2..4 */
    int32_t ntiles;           /* 24 (no jokers) or 26 */
    int32_t deal;             /* tiles dealt to each player (Sec. II-A: 4) */
    int32_t max_predraw;      /* root generation: post-deal draws uniform in 0..max_predraw */
    int32_t max_revealed;     /* root generation: reject histories with more face-up tiles per player */
    uint32_t cont_thr;        /* see above */
    double c_uct;             /* sqrt(2); UCB1 runs in IEEE single precision with c rounded to float */
    int32_t d_max;            /* 8 */
    int32_t playouts;         /* playouts per leaf in dvc_mcts_step (leaf parallelism) */
    int32_t policy;           /* playout guesses: 0 uniform (default), 1 ordering-aware (see above) */
    int32_t tree_continue;    /* 0: the simplified tree (default); 1: the full game tree (see above) */
    int32_t vanilla;          /* 0: MCTS-dvc (default); 1: plausible-set root children (see above) */
} dvc_config;

typedef struct dvc_ctx dvc_ctx;
typedef struct dvc_forest dvc_forest;

/* Create a context on CUDA device `device` with a copy of *cfg.  Validates
 * the configuration (DVC_E_INVALID).  Owns nothing on the device until a
 * call needs workspace. */
int dvc_create(dvc_ctx** out, const dvc_config* cfg, int device);
void dvc_destroy(dvc_ctx* ctx);
const char* dvc_last_error(const dvc_ctx* ctx);

/* Synchronise the context's device and report (then clear) any error a
 * kernel latched: DVC_E_UNSUPPORTED, DVC_E_OOM, DVC_E_TIMEOUT, or
 * DVC_E_INVALID for an illegal guess passed to dvc_play_move. */
int dvc_check(dvc_ctx* ctx);

/*
 * Root states (Sec. II-A deal; the workload's mid-game roots).  State i is
 * generated on its own stream (seed, tree id i, tag 1): a deal of cfg->deal
 * tiles to each seat in order, a random-policy history of d post-deal draws
 * with d uniform in 0..max_predraw, then the seat to move draws.  Histories
 * that end the game or leave a seat with more than max_revealed face-up
 * tiles are retried on the same stream (16 attempts; the last uses d = 0).
 * d_states: n records, written.  n = 0 is a no-op.
 */
int dvc_init_states(dvc_ctx* ctx, uint64_t seed, int n, dvc_state* d_states, void* stream);

/*
 * Determinization (Sec. III-A, plausible numbers): for each root r, a fresh
 * assignment of the tiles `observer` cannot see, drawn uniformly among all
 * assignments consistent with its view -- each opponent's slot count, face-up
 * tiles in place, numbered tiles ascending, jokers free -- on the stream
 * (seed, d_tree_ids[r], iteration d_iter_ids[r], tag 2).  observer < 0 means
 * each root's seat to move.  d_roots and d_out: n records (may not overlap);
 * d_tree_ids, d_iter_ids: n uint32 each.  A view whose counting table exceeds
 * 32768 cells latches DVC_E_UNSUPPORTED (see dvc_check) and leaves that
 * output equal to its root.
 */
int dvc_determinize(dvc_ctx* ctx, const dvc_state* d_roots, int n, int observer, uint64_t seed,
                    const uint32_t* d_tree_ids, const uint32_t* d_iter_ids, dvc_state* d_out, void* stream);

/*
 * Leaf-parallel random playouts (Sec. II-B simulation; Sec. III-D: every GPU
 * thread plays games out to a win or loss).  For leaf l and j in
 * 0..playouts_per_leaf-1, playout j runs on stream (seed, d_tree_ids[l],
 * playout j, leaf d_leaf_ids[l], tag 4) from d_leaves[l] (seat to move about
 * to guess) with uniform guesses, cfg->cont_thr, until one seat is left.
 * d_wins: n_leaves x 4 int32, OVERWRITTEN with the number of playouts each
 * seat won (a finished leaf credits all playouts to its winner).
 * d_words (optional, may be NULL): one uint64, overwritten with the number of
 * random words the playouts consumed (the work count behind the roofline).
 */
int dvc_rollout_batch(dvc_ctx* ctx, const dvc_state* d_leaves, int n_leaves, int playouts_per_leaf, uint64_t seed,
                      const uint32_t* d_tree_ids, const uint32_t* d_leaf_ids, int32_t* d_wins, uint64_t* d_words,
                      void* stream);

/*
 * One move of each of n games played out by search agents (self-play; the
 * game model the tree searches, Sec. III-A simplification 2): the seat to
 * move in d_states[i] makes the guess d_actions[i] (action code seat << 10 |
 * slot << 5 | identity, as dvc_root_stats reports it) on the true state; the
 * turn ends after the guess, correct or not; then the next seat still in
 * draws on stream (seed, d_game_ids[i] or i if NULL, turn, tag 5).  d_states
 * is updated in place; d_actions[i] < 0 or a finished game leaves the record
 * unchanged.  An illegal guess leaves the record unchanged and latches
 * DVC_E_INVALID (see dvc_check).  All pointers are device memory.
 */
int dvc_play_move(dvc_ctx* ctx, dvc_state* d_states, int n, const int32_t* d_actions, uint64_t seed,
                  const uint32_t* d_game_ids, uint32_t turn, void* stream);

/*
 * A forest of independent UCT trees (Sec. II-B; Sec. III-B runs many at
 * once).  Tree t searches from d_roots[t] for the seat to move there, with
 * h_budgets[t] iterations (one node per iteration at most; 0..2^24) and
 * streams keyed (seed, h_tree_ids ? h_tree_ids[t] : t).  d_roots is copied
 * on `stream`; h_budgets and h_tree_ids are host arrays read during the call.
 * Device memory per tree: a node arena of 641 + 4 * budget 36-byte slots
 * (node 16 B, cached UCB1 terms 12 B, child link 4 B, creation stamp 4 B;
 * vanilla: 1 + 5 * budget slots, plus a plausible-set table of 2 * budget
 * 20-byte cells), a
 * determinization table of 2,048 cells (2 players) or 32,768 cells (3-4
 * players) of 8 bytes, and 64 determinized roots with the first block of
 * their in-tree random streams (3 KB) sampled ahead by both engines.  The root
 * views are planned on the device without a host synchronisation; a view
 * whose table does not fit latches
 * DVC_E_UNSUPPORTED and its tree does no work.  DVC_E_OOM if memory runs out.
 */
int dvc_forest_create(dvc_ctx* ctx, int n_trees, const dvc_state* d_roots, const int32_t* h_budgets,
                      const uint32_t* h_tree_ids, uint64_t seed, dvc_forest** out, void* stream);
void dvc_forest_destroy(dvc_forest* f);

/* Start every tree of the forest afresh (budgets, tree ids and seed kept):
 * with d_roots non-NULL the forest first copies n_trees new roots from it.
 * Asynchronous on `stream`; allocates nothing. */
int dvc_forest_reset(dvc_forest* f, const dvc_state* d_roots, void* stream);

/*
 * Fused search step: every tree runs min(n_iterations, budget - done)
 * iterations of: determinize the root view (tag 2, iteration i), descend by
 * UCB1 -- score = wins/n + (c_uct * sqrt(ln N)) * (1/sqrt(n)), N the parent's
 * visits, ln by the library's own argument-reduced atanh series, ties to the
 * lowest canonical action -- among children legal in this determinization,
 * expand the first legal action without a child (canonical order: opponents
 * from cur+1, slots left to right, identities ascending) while the depth is
 * below d_max, draw in-tree tiles on tag 3, score the leaf (mode ROLLOUT:
 * cfg->playouts playouts on tag 4 keyed by iteration; mode VALUE: the value
 * network of the context, see dvc_value_eval, credits each seat
 * round(p * cfg->playouts) of the cfg->playouts visits; a leaf that ended in
 * the tree credits its winner in both modes), and add cfg->playouts visits
 * and each node's mover's wins along the path.  Rollout results are
 * bit-exact with the split steps for every engine and launch shape.
 */
int dvc_mcts_step(dvc_forest* f, int n_iterations, int mode, void* stream);

/*
 * Engine and launch shape of dvc_mcts_step (no effect on results).
 * engine 1: one fused kernel; each CTA runs trees_per_cta trees in lockstep
 * with warps_per_cta warps (every warp walks a tree, then all lanes share the
 * leaves' playouts; every 64 iterations all threads sample the next 64
 * determinizations of every tree, one thread each).  engine 2: per iteration two launches (backprop of the
 * previous iteration + select, then pooled rollouts) in a CUDA graph of 64
 * iterations; rollout CTAs pool trees_per_cta trees with warps_per_cta warps,
 * and the CTAs are split into `chains` (1..32) independent chains on
 * separate streams so that one chain's tree walks run beside another chain's
 * playouts.  The determinizations of the graph's 64 iterations are sampled
 * up front, one thread per tree and iteration.  engine 0 keeps the current
 * engine (the default is 2 for forests of more than four trees per SM, else 1).
 * trees_per_cta, warps_per_cta, chains 0 = the engine's defaults (fused:
 * ceil(n_trees / SMs) trees, at most 32, and a warp per tree or one playout
 * per thread, whichever is more, up to 16 warps;
 * pipeline: round(n_trees / (1.12 SMs)) chains, at most 24; at least 2 trees,
 * ceil(n_trees / (0.85 chains SMs)), at most 64; warps for one playout per
 * thread, 4 to 16).  Changing
 * trees_per_cta re-balances which trees share a CTA (longest budget first,
 * least-loaded CTA; equal budgets keep index order) and synchronises the
 * device once.  DVC_E_UNSUPPORTED if
 * a CTA's state would not fit in shared memory.
 */
int dvc_forest_tune(dvc_forest* f, int engine, int trees_per_cta, int warps_per_cta, int chains);

/*
 * Which trees share a CTA, set by the caller: h_order (host, n_trees int32)
 * is a permutation of 0 .. n_trees-1; CTA b of either engine takes the trees
 * h_order[b * trees_per_cta ..].  n_active (0 .. n_trees; 0 = all) limits the
 * fused engine's launches to the first n_active trees of the order -- a caller
 * that knows which trees still have iterations left lists those first and
 * packs trees of similar remaining budgets together; the other trees must have
 * no iterations left in the steps that follow (they are not visited).  Results
 * are identical for every order.  The next dvc_forest_tune that changes
 * trees_per_cta replaces the order and, like dvc_forest_reset, clears
 * n_active (all trees run); h_order NULL (n_active 0) restores the default
 * order of the current CTA size.  Synchronises the device once.
 * DVC_E_INVALID if h_order is not a permutation or n_active is out of range.
 */
int dvc_forest_order(dvc_forest* f, const int32_t* h_order, int n_active);

/*
 * The same iteration split into launches, for callers that score leaves
 * themselves: dvc_mcts_select determinizes and descends, dvc_mcts_expand adds
 * the new child and writes each tree's leaf state (dvc_forest_leaves gives
 * the device pointer, n_trees records; trees whose budget is spent are
 * marked finished with winner = 0xFE), the caller fills n_trees x 4 int32
 * wins (e.g. with dvc_rollout_batch, tree ids and leaf ids from
 * dvc_forest_leaf_ids), and dvc_mcts_backprop adds them.
 */
int dvc_mcts_select(dvc_forest* f, void* stream);
int dvc_mcts_expand(dvc_forest* f, void* stream);
int dvc_mcts_backprop(dvc_forest* f, const int32_t* d_wins, void* stream);
int dvc_forest_leaves(dvc_forest* f, dvc_state** d_leaves, uint32_t** d_tree_ids, uint32_t** d_leaf_ids);

/*
 * Root statistics and decision (Sec. III-B merge, one tree): per tree 8 int32
 * -- best action (most visits, ties to the lowest canonical action; -1 if
 * none), its visits, its wins, root visits, root children, nodes used,
 * iterations done, 0.  Action code = seat << 10 | slot << 5 | identity.
 * Vanilla trees: an action's visits and wins are summed over the plausible
 * sets, and root children counts the sets.  d_out: n_trees x 8 int32.
 */
int dvc_root_stats(dvc_forest* f, int32_t* d_out, void* stream);

/*
 * Root-parallel merge (Sec. III-B: independent searches of one position
 * whose root statistics are summed, the paper's "amalgamated" trees).  The
 * forest's trees form n / K groups of K consecutive trees; the trees of a
 * group must share their root (their streams differ through their tree ids;
 * a group whose roots differ latches DVC_E_INVALID).  Per group, 8 int32:
 * the action with the most visits summed over the group (for vanilla trees
 * summed over every plausible set as well), ties to the lowest canonical
 * action (-1 if none); its summed visits; its summed wins (the searching
 * seat's); the summed root visits; the number of distinct root actions; K;
 * the summed iterations done; 1 if any tree failed.  d_out: n / K x 8
 * int32.  DVC_E_INVALID unless K divides the number of trees;
 * DVC_E_UNSUPPORTED if K x budget x playouts could exceed 2^31.
 */
int dvc_root_merge(dvc_forest* f, int K, int32_t* d_out, void* stream);

/* Work counters of the forest since creation or the last call: d_out[0] =
 * random words consumed by its playouts (each word is one uniform choice of
 * the method: a draw, a joker position, a guess or a continue coin).  Copies
 * then zeroes the counter, on `stream`.  d_out: one uint64. */
int dvc_forest_counters(dvc_forest* f, uint64_t* d_out, void* stream);
/* Lane compaction in the pipeline engine's two-player 24-tile playouts
 * (uniform policy, no may-stop leaves; other forests ignore it), off by
 * default (receivers = 0).  The paper studies the branch divergence of GPU
 * playouts (Sec. IV); this regroups running games instead: once a rollout
 * CTA's pool of playouts is empty, each of its warps from `receivers` on
 * that has at most `donate_at` games running hands them (state and stream
 * position) to the CTA's first `receivers` warps, whose idle lanes finish
 * them.  Results are identical either way.  DVC_E_INVALID unless
 * 0 <= receivers < warps per rollout CTA and 1 <= donate_at <= 31.  Takes
 * effect at the next dvc_mcts_step. */
int dvc_forest_compaction(dvc_forest* f, int receivers, int donate_at);
/* The forest's playout work since creation or the last call, two uint64:
 * d_out[0] random words (as dvc_forest_counters), d_out[1] game steps -- one
 * per guess of a playout (Sec. II-A: the guess with its resolution, any
 * continue coin and the next seat's draw), plus one for the continue coin a
 * playout from a may-stop leaf draws first.  Copies then zeroes both
 * counters, on `stream`. */
int dvc_forest_work(dvc_forest* f, uint64_t* d_out, void* stream);
/* Work counting (dvc_forest_counters, dvc_forest_work) on (the default) or
 * off.  The counts are instrumentation, not part of the search: off, the
 * playout kernels keep no counts (the two-player 24-tile playout kernel
 * then runs a counting-free variant, about 1.5 % faster) and both counters
 * keep their values; results are identical either way.  Takes effect at the
 * next dvc_mcts_step.  DVC_E_INVALID for a null forest. */
int dvc_forest_count_work(dvc_forest* f, int on);

/* Nodes of tree t in creation order, 4 int32 each: action, parent (-1 for
 * the root), visits, wins.  d_out holds h_budgets[t] + 1 rows; rows past the
 * nodes used are set to -1. */
int dvc_tree_export(dvc_forest* f, int tree, int32_t* d_out, void* stream);

/*
 * dvc_determinize without any allocation, for callers that cannot call
 * cudaMalloc: a process whose device memory is fully reserved by another
 * framework's caching allocator, or one that may not allocate after start-up.
 * The paper has no counterpart; this is a deployment variant of
 * dvc_determinize.  For views whose counting table fits 16,384 cells and an
 * observer below each root's player count (or -1, the seat to move) it
 * returns the same records as dvc_determinize for the same arguments.
 * It needs no context: it runs on the calling thread's current device, and
 * every pointer must be memory of that device (or managed memory); any other
 * pointer, or d_out overlapping d_roots, returns DVC_E_INVALID and enqueues
 * nothing.  Its scratch is a fixed 8 MiB device array inside the library
 * (64 roots x 16,384 table cells), held by every GPU that loads the library
 * until exit.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents
 * (nothing in it needs to start at zero); calls that overlap on the GPU race
 * on it, so issue them on one stream.  n > 64 returns DVC_E_UNSUPPORTED and
 * enqueues nothing.  d_status (optional, n int32) per root: 0; DVC_E_INVALID
 * when observer >= that root's player count (dvc_determinize refuses such a
 * call on the host); DVC_E_UNSUPPORTED for a view whose table needs more
 * than 16,384 cells (dvc_determinize handles up to 32,768).  In both error
 * cases that output record is the root itself.  Calls no cudaMalloc or
 * cudaFree.
 */
int dvc_determinize_noalloc(const dvc_state* d_roots, int n, int observer, uint64_t seed,
                            const uint32_t* d_tree_ids, const uint32_t* d_iter_ids, dvc_state* d_out,
                            int32_t* d_status, void* stream);

/*
 * Value network: a learned leaf evaluator that can replace playouts (the
 * workload's extension; the paper's own leaf evaluation is the random playout
 * of Sec. II-B).  Features (640, BF16): per tile the owner seat relative to the
 * mover, face down/up and drawn this turn; per opponent slot the values it may
 * hold given its face-up numbered neighbours and the tiles the mover cannot
 * see.  640 -> 512 -> 512 -> 512 (GELU) -> 4 logits over relative seats,
 * softmax over the seats in play.  BF16 weights and activations with FP32
 * accumulation on the tensor cores (tcgen05, accumulators in tensor memory);
 * FP32 master weights and AdamW moments.  Parameters, as a flat FP32 array:
 * W1[512][640], b1[512], W2[512][512], b2[512], W3[512][512], b3[512],
 * W4[4][512], b4[4] (855,556 values).  The network lives in the context.
 */
/* Initialise the weights (Glorot uniform from Philox keyed by seed; zero biases). */
int dvc_value_init(dvc_ctx* ctx, uint64_t seed, void* stream);
/* Copy the FP32 parameters out (direction 0) or in (direction 1); d_params: 855,556 floats. */
int dvc_value_params(dvc_ctx* ctx, float* d_params, int direction, void* stream);
/* Features of n states, FP32 0/1, n x 640 (test and inspection hook). */
int dvc_value_features(dvc_ctx* ctx, const dvc_state* d_states, int n, float* d_out, void* stream);
/* Win probability per absolute seat for n leaves: d_winprob n x 4 FP32 (seats beyond the game's player count 0). */
int dvc_value_eval(dvc_ctx* ctx, const dvc_state* d_leaves, int n, float* d_winprob, void* stream);
/* One AdamW step (beta 0.9/0.999, eps 1e-8, weight decay 1e-4 on matrices) on the
 * mean cross-entropy of n states against soft labels d_labels (n x 4 FP32, per
 * absolute seat, summing to 1).  d_loss (optional): the mean loss before the step. */
int dvc_value_train_step(dvc_ctx* ctx, const dvc_state* d_states, const float* d_labels, int n, float lr,
                         float* d_loss, void* stream);
/* Gradient of the last train step (855,556 FP32, parameter layout above). */
int dvc_value_grads(dvc_ctx* ctx, float* d_out, void* stream);
/* Checkpoint: weights, AdamW moments and step, to and from a host file (synchronises). */
int dvc_value_save(dvc_ctx* ctx, const char* path);
int dvc_value_load(dvc_ctx* ctx, const char* path);
/* The tensor-core GEMM used by the network: C = act(A B^T + bias), A M x K and
 * B N x K row-major BF16, bias N FP32 (optional), C M x N BF16 (optional),
 * Cf M x N FP32 before the activation (optional); N % 16 == 0, K % 64 == 0;
 * act 0 none, 1 GELU (tanh form); all pointers 16-byte aligned
 * (DVC_E_INVALID otherwise). */
int dvc_gemm_bf16(dvc_ctx* ctx, const void* d_A, const void* d_B, const float* d_bias, void* d_C, float* d_Cf, int M,
                  int N, int K, int act, void* stream);
/* Test hook of the GEMM's failure path (not part of the method): the same
 * kernel with its copy-issuing warp issuing nothing, so the tensor-core and
 * epilogue warps' mbarrier waits run out after wait_ms (1..1000) with no copy
 * or MMA in flight; the kernel frees its tensor memory, exits and latches
 * DVC_E_TIMEOUT, which dvc_check reports.  d_Cf is not written.  Every
 * mbarrier wait of the GEMM is bounded this way (2 s in normal calls). */
int dvc_gemm_timeout_probe(dvc_ctx* ctx, const void* d_A, const void* d_B, float* d_Cf, int M, int N, int K,
                           int wait_ms, void* stream);

/*
 * Serving: a request loop that keeps many searches resident on the device.
 * Move queries from concurrent games (root state, iteration budget, leaf
 * mode, id) wait in a FIFO queue and are admitted as search slots free up
 * (continuous batching).  The slots form lanes (below); each lane steps on
 * its own stream: a step runs `iterations` more iterations of every resident
 * search of the lane together.  A poll collects the lanes whose step has
 * finished (returning the queries whose budget is complete), admits queued
 * queries into their free slots and starts their next step; if no lane had
 * finished it waits (on the host) until one has.  Slots are sized for
 * max_budget iterations and their number is fixed at creation by the HBM
 * budget, so admission is by memory.  A query's search is keyed by (seed,
 * low 32 bits of its id) and runs exactly as it would alone: results do not
 * depend on what else is resident.  Host-side calls; poll synchronises the
 * server's own streams.  A vanilla context returns DVC_E_UNSUPPORTED.
 *
 * A server may hold several game variants (player count and tile set), one
 * context each: its slots are split into lanes, one per (context, leaf mode),
 * each a forest of that variant with its own stream, so the searches of
 * different variants and modes run side by side on the GPU.  A submitted
 * root goes to the lane of its variant and mode.  CUDA maps streams onto
 * CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 by default): for the lanes
 * of a larger server to run side by side, raise it (e.g. to 32) before the
 * process's first CUDA call.  The paper searches one game at a time; serving
 * many games is not part of its method.
 */
typedef struct dvc_server dvc_server;
typedef struct dvc_result {
    uint64_t query_id;
    int32_t best_action, best_visits, best_wins, root_visits, iterations, mode;
    double t_submit, t_done; /* host steady-clock seconds */
} dvc_result;
/* One context.  value_share_pct of the budget goes to value-mode slots if
 * the context has a value network. */
int dvc_server_create(dvc_ctx* ctx, size_t hbm_budget, int max_budget, int value_share_pct, uint64_t seed,
                      dvc_server** out);
/* n_ctx (1..16) contexts of distinct game variants on one device.  Context i
 * gets h_weights[i] / sum(h_weights) of hbm_budget (NULL: equal shares),
 * value_share_pct of that for value-mode slots if it has a value network;
 * its slot count is that share over its per-slot footprint (node arena for
 * max_budget iterations, counting table, buffers).  Each context's value
 * network serves its own variant's value-mode queries.  DVC_E_INVALID for
 * two contexts of one variant or contexts on different devices; DVC_E_OOM if
 * the budget holds no slot at all. */
int dvc_server_create_multi(dvc_ctx* const* ctxs, int n_ctx, const int32_t* h_weights, size_t hbm_budget,
                            int max_budget, int value_share_pct, uint64_t seed, dvc_server** out);
void dvc_server_destroy(dvc_server* sv);
/* Queue a query; h_root is a host record of one of the server's variants
 * (DVC_E_INVALID otherwise; DVC_E_UNSUPPORTED if that variant has no slots
 * of this mode). */
int dvc_server_submit(dvc_server* sv, const dvc_state* h_root, int budget, int mode, uint64_t query_id);
/* Collect finished lanes, admit, start their next `iterations`; returns the number of results written
 * (<= max_results; results that did not fit are returned by the next poll). */
int dvc_server_poll(dvc_server* sv, int iterations, dvc_result* h_results, int max_results);
/* h_out[5]: queued, resident, completed, rollout slots, value slots (over all lanes). */
int dvc_server_stats(dvc_server* sv, int64_t* h_out);
/* Per lane, 8 int32: context index, players, tiles, mode, slots, resident,
 * steps collected so far, their mean device time in microseconds (from the
 * step's first launch to its statistics on the host side of the copy).
 * Writes min(lanes, max_lanes) rows; returns the number of lanes. */
int dvc_server_lanes(dvc_server* sv, int max_lanes, int32_t* h_out);

/* Test hook for the random-number generator: out[4k..4k+3] = Philox-4x32-10
 * of counter d_ctr[4k..], key d_key[2k..], by this library's generator
 * (use_reference = 0) or by cuRAND's device function (use_reference = 1). */
int dvc_philox(dvc_ctx* ctx, int n, const uint32_t* d_ctr, const uint32_t* d_key, uint32_t* d_out,
               int use_reference, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DVC_H */
