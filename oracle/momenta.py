"""Momentum list for the p^2 cut (Sec. 2.1.1 "up to p^2 <= 9", Sec. 2.3).

Reading: p = 2 pi n / L with integer n = (nx, ny, nz) and the cut applies to
n^2 = nx^2 + ny^2 + nz^2 <= p2max.  Order: ascending n^2, ties by ascending
lexicographic (nx, ny, nz).  Found here by brute-force enumeration of the
cube |n_i| <= p2max and sorting with that key.
"""


def momentum_list(p2max=9):
    r = 0
    while (r + 1) * (r + 1) <= p2max:
        r += 1
    out = []
    for nx in range(-r, r + 1):
        for ny in range(-r, r + 1):
            for nz in range(-r, r + 1):
                n2 = nx * nx + ny * ny + nz * nz
                if n2 <= p2max:
                    out.append((n2, nx, ny, nz))
    out.sort()
    return [(nx, ny, nz) for (_, nx, ny, nz) in out]
