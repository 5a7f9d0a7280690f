"""D2Q9 velocity set (Sec. 2, the paragraph introducing Eq. extendedFeq).

Discrete velocities have components xi_{i,alpha} in {0, +1, -1}; the lattice is the
tensor product of two D1Q3 lattices.  The lattice constant (isothermal temperature) is
c_s^2 = T_0 = 1/3 (used in Eq. extendedFeq, in omega_nu of Sec. 4c and in App. B).

Population index convention (shared by oracle and GPU as an interface, not as code):
  i : 0      1      2      3       4       5      6       7        8
  xi: (0,0)  (1,0)  (0,1)  (-1,0)  (0,-1)  (1,1)  (-1,1)  (-1,-1)  (1,-1)
"""

import numpy as np

Q = 9
XI = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
               [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
CS2 = 1.0 / 3.0

# the nine moment indices (p, q) with p, q <= 2 used throughout App. B
PQ = [(p, q) for p in range(3) for q in range(3)]


def index_of(sx, sy):
    """Population index i whose velocity is (sx, sy)."""
    for i in range(Q):
        if XI[i, 0] == sx and XI[i, 1] == sy:
            return i
    raise ValueError((sx, sy))
