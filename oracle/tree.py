"""Index tree of Section 3.1 ("A tree structure") -- oracle side.

Test infrastructure only (see ``oracle/__init__.py``).

Readings taken where the paper is loose:
* a node is split while its size exceeds the leaf threshold ``m`` ("below some given
  threshold", Section 3.1, read as "at most m", matching "maximum leaf node size" of Section 5);
* the left child receives the first ceil(n/2) indices (Section 3.1);
* the tree is fully populated: every node of a level is split together, so all leaves sit
  on level L (Section 3.1, last paragraph);
* nodes are numbered as in Fig. 1: root 1, children of tau are 2 tau and 2 tau + 1, so level l
  holds nodes 2^l .. 2^(l+1) - 1 from left to right.
Offsets are 0-based (I_tau = [offset, offset + size)).
"""


def tree_depth(N, leaf_max):
    """Depth L: the first level at which every node holds at most ``leaf_max`` indices.

    Splits are done by brute force (no closed form), exactly as Section 3.1 describes.
    """
    if N < 1 or leaf_max < 1:
        raise ValueError("N and leaf_max must be positive")
    sizes = [N]
    L = 0
    while max(sizes) > leaf_max:
        nxt = []
        for n in sizes:
            left = (n + 1) // 2          # ceil(n / 2) goes to the left child
            nxt += [left, n - left]
        sizes = nxt
        L += 1
    return L


def build_tree(N, leaf_max):
    """Return (L, offsets, sizes) with lists indexed by node id 1 .. 2^(L+1) - 1 (entry 0 unused).

    Section 3.1: root gets [0, N); each parent [o, o + n) gives [o, o + ceil(n/2)) to its left
    child and the rest to its right child; splitting stops at depth L (``tree_depth``).
    """
    L = tree_depth(N, leaf_max)
    count = 2 ** (L + 1)
    offsets = [0] * count
    sizes = [0] * count
    offsets[1], sizes[1] = 0, N
    for tau in range(1, 2 ** L):
        n, o = sizes[tau], offsets[tau]
        left = (n + 1) // 2
        offsets[2 * tau], sizes[2 * tau] = o, left
        offsets[2 * tau + 1], sizes[2 * tau + 1] = o + left, n - left
    return L, offsets, sizes


def level_nodes(level):
    """Node ids on ``level`` (Fig. 1 numbering), left to right."""
    return list(range(2 ** level, 2 ** (level + 1)))


def children(tau):
    """(alpha, beta): left and right child of ``tau`` (Fig. 1 numbering)."""
    return 2 * tau, 2 * tau + 1
