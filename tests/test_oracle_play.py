"""Pins for the oracle's self-play move (one guess of the tree model, Sec.
III-A, then the next seat's draw) and its canonical legal-action list."""
import numpy as np
import pytest

import oracle
from statefmt import decode, encode

SEED, GAME, TURN = 0x1234_0000_0007, 11, 5


def _draw_word():
    """First word of the play stream: Philox-4x32-10 of counter (block 0,
    j 0, turn, tag 5 + 16 * high seed word), key (low seed word, game)."""
    lo, hi = SEED & 0xFFFFFFFF, SEED >> 32
    return oracle.philox4x32_10([0, 0, TURN, 5 + 16 * hi], [lo, GAME])[0]


def _expected_draw(hands, ntiles=24):
    held = {t for h in hands for t in h}
    pool = [t for t in range(ntiles) if t not in held]
    return pool[(_draw_word() * len(pool)) >> 32]


# player 0 to move holds 1, 6 (drawn) and 14 (face up); player 1 holds 3, 10 (face up), 17
HANDS = [[1, 6, 14], [3, 10, 17]]
REV = {10, 14}


def _pos():
    return encode(HANDS, REV, cur=0, drawn=6, ntiles=24)


def test_legal_actions_canonical_order():
    codes = oracle.legal_actions(_pos())
    ids = [x for x in range(24) if x not in (1, 6, 14, 10)]          # not own, not face up
    want = [(1 << 10) | (0 << 5) | x for x in ids] + [(1 << 10) | (2 << 5) | x for x in ids]
    assert codes.tolist() == want
    pre = encode([[0, 2, 4, 6], [1, 3, 5, 7]], set(), cur=0, drawn=None, ntiles=26)
    assert len(oracle.legal_actions(pre)) == 88 == oracle.legal_count(pre)   # Sec. III-A


def test_correct_guess_ends_turn_and_next_seat_draws():
    rc, out = oracle.play_move(_pos(), (1 << 10) | (0 << 5) | 3, SEED, GAME, TURN)
    assert rc == 0
    d = decode(out)
    t = _expected_draw(HANDS)
    assert d["revealed"] == REV | {3}
    assert d["cur"] == 1 and d["drawn"] == t and d["winner"] is None
    assert d["hands"][1] == sorted([3, 10, 17, t]) and d["hands"][0] == [1, 6, 14]


def test_wrong_guess_reveals_drawn_tile():
    rc, out = oracle.play_move(_pos(), (1 << 10) | (2 << 5) | 18, SEED, GAME, TURN)
    assert rc == 0
    d = decode(out)
    assert d["revealed"] == REV | {6}
    assert d["cur"] == 1 and d["drawn"] == _expected_draw(HANDS)


def test_eliminations_end_the_game():
    # correct guess at the opponent's last face-down tile: the guesser wins, nobody draws
    s = encode([[1, 6], [3, 10]], {10}, cur=0, drawn=6, ntiles=24)
    rc, out = oracle.play_move(s, (1 << 10) | (0 << 5) | 3, SEED, GAME, TURN)
    d = decode(out)
    assert rc == 0 and d["winner"] == 0 and d["revealed"] == {3, 10} and d["hands"][0] == [1, 6]
    # wrong guess with only the drawn tile face down: the guesser is out, the opponent wins
    s = encode([[1, 6], [3, 10]], {1}, cur=0, drawn=6, ntiles=24)
    rc, out = oracle.play_move(s, (1 << 10) | (1 << 5) | 11, SEED, GAME, TURN)
    d = decode(out)
    assert rc == 0 and d["winner"] == 1 and d["revealed"] == {1, 6}


def test_empty_pool_and_leftmost_reveal():
    # all 24 tiles held: a wrong guess with nothing drawn reveals the leftmost
    # face-down tile, and the next seat has nothing to draw
    h0 = list(range(0, 24, 2))
    h1 = list(range(1, 24, 2))
    s = encode([h0, h1], {0}, cur=0, drawn=None, ntiles=24)
    rc, out = oracle.play_move(s, (1 << 10) | (0 << 5) | 5, SEED, GAME, TURN)   # slot 0 holds 1, not 5
    d = decode(out)
    assert rc == 0 and d["revealed"] == {0, 2} and d["cur"] == 1 and d["drawn"] is None


def test_illegal_and_finished():
    s = _pos()
    for code in (-1, (0 << 10) | 3, (1 << 10) | (1 << 5) | 3, (1 << 10) | (0 << 5) | 14, (1 << 10) | (5 << 5) | 3):
        rc, out = oracle.play_move(s, code, SEED, GAME, TURN)
        assert rc == -1 and (out == s).all(), code
    over = encode(HANDS, REV | {3, 17}, cur=0, drawn=6, ntiles=24, winner=0)
    rc, out = oracle.play_move(over, (1 << 10) | 3, SEED, GAME, TURN)
    assert rc == 1 and (out == over).all()
