"""Test-side encoder/decoder of the 32-byte state record (format only).

Builds records from explicit hands so tests can pose hand-made positions to
both the oracle and the GPU library, and decodes records back to hands for
invariant checks.  No game rule lives here.

Layout: hand[4] u32 tile bitmasks (bytes 0..15), revealed u32 (16..19),
joker gaps u8[2] (20, 21: numbered tiles left of joker 24 / 25 in its owner's
hand), flags u8 (22, bit 0: jokers share owner and gap and 25 comes first;
bit 1: the player to move guessed correctly this turn and may stop),
cur (23), drawn (24, 0xFF none), alive mask (25), players (26), tiles (27),
winner (28, 0xFF running), padding (29..31).
"""
import numpy as np

JB, JW = 24, 25


def encode(hands, revealed, cur, drawn=None, ntiles=24, alive=None, winner=None, may_stop=False):
    """hands: list of per-player left-to-right tile-id lists; revealed: set of ids."""
    P = len(hands)
    b = np.zeros(32, dtype=np.uint8)
    for p, h in enumerate(hands):
        m = 0
        for t in h:
            m |= 1 << t
        b[4 * p:4 * p + 4] = np.frombuffer(np.uint32(m).tobytes(), dtype=np.uint8)
    rv = 0
    for t in revealed:
        rv |= 1 << t
    b[16:20] = np.frombuffer(np.uint32(rv).tobytes(), dtype=np.uint8)
    owner = {}
    pos = {}
    for p, h in enumerate(hands):
        for i, t in enumerate(h):
            owner[t] = p
            pos[t] = i
    for j, t in enumerate((JB, JW)):
        if t in owner:
            h = hands[owner[t]]
            b[20 + j] = sum(1 for u in h[:pos[t]] if u < 24)
    if JB in owner and JW in owner and owner[JB] == owner[JW] and b[20] == b[21] and pos[JW] < pos[JB]:
        b[22] = 1
    if may_stop:
        b[22] |= 2
    b[23] = cur
    b[24] = 0xFF if drawn is None else drawn
    if alive is None:
        alive = [any(t not in revealed for t in h) for h in hands]
    b[25] = sum(1 << p for p, a in enumerate(alive) if a)
    b[26] = P
    b[27] = ntiles
    b[28] = 0xFF if winner is None else winner
    return b


def decode(b):
    """Returns dict with hands (left-to-right lists), revealed set, cur, drawn,
    alive list, P, T, winner."""
    b = np.asarray(b, dtype=np.uint8).reshape(32)
    P, T = int(b[26]), int(b[27])
    masks = [int(np.frombuffer(b[4 * p:4 * p + 4].tobytes(), dtype=np.uint32)[0]) for p in range(4)]
    rv = int(np.frombuffer(b[16:20].tobytes(), dtype=np.uint32)[0])
    hands = []
    for p in range(P):
        m = masks[p]
        num = [t for t in range(24) if m >> t & 1]
        seq = []
        order = (JW, JB) if b[22] & 1 else (JB, JW)
        for g in range(len(num) + 1):
            for t in order:
                if m >> t & 1 and b[20 + t - JB] == g:
                    seq.append(t)
            if g < len(num):
                seq.append(num[g])
        hands.append(seq)
    return {
        "hands": hands,
        "masks": masks,
        "revealed": {t for t in range(32) if rv >> t & 1},
        "cur": int(b[23]),
        "drawn": None if b[24] == 0xFF else int(b[24]),
        "alive": [bool(b[25] >> p & 1) for p in range(P)],
        "P": P,
        "T": T,
        "winner": None if b[28] == 0xFF else int(b[28]),
        "may_stop": bool(b[22] & 2),
    }
