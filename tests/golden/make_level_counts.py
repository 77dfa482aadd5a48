"""Write level_cell_counts.txt: boxes of the n^3 grid over [-1,1]^3 meeting the
closed unit ball, by exact integer arithmetic.

With h = 2/n the box of index i spans [-1 + i h, -1 + (i+1) h]; in units of
h/2 = 1/n its bounds are the integers 2i - n and 2i + 2 - n, so the squared
distance from the origin to the box, times n^2, is an integer. The box meets
the ball iff that integer sum is <= n^2.  Nothing here uses the oracle.
"""
import os


def dist_units(i: int, n: int) -> int:
    lo, hi = 2 * i - n, 2 * i + 2 - n
    if lo > 0:
        return lo
    if hi < 0:
        return -hi
    return 0


def count(n: int) -> int:
    d2 = [dist_units(i, n) ** 2 for i in range(n)]
    lim = n * n
    tot = 0
    for z in range(n):
        for y in range(n):
            r = lim - d2[z] - d2[y]
            if r < 0:
                continue
            tot += sum(1 for x in range(n) if d2[x] <= r)
    return tot


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "level_cell_counts.txt"), "w") as f:
        f.write("# n  cells-meeting-closed-unit-ball  (exact integer lattice count, make_level_counts.py)\n")
        for n in (2, 4, 8, 16, 32, 64, 128):
            f.write(f"{n} {count(n)}\n")
