"""Writes select_tables.inc: for every 12-bit value, the positions of its set
bits, 4 bits per rank (rank r in bits 4r..4r+3), as a u64.  Used by the
playout kernels to find the n-th set bit of a tile mask with one lookup per
12-bit half."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    vals = []
    for v in range(4096):
        w, r = 0, 0
        for b in range(12):
            if v >> b & 1:
                w |= b << (4 * r)
                r += 1
        vals.append(w)
    with open(os.path.join(HERE, "..", "select_tables.inc"), "w") as f:
        f.write("// generated by gen/select_tables.py\n")
        for i in range(0, 4096, 4):
            f.write(", ".join("0x%016Xull" % x for x in vals[i:i + 4]) + ",\n")


if __name__ == "__main__":
    main()
