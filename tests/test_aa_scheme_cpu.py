"""Race freedom of the in-place AA streaming scheme, checked on the CPU by
brute force over its access pattern (racecheck is not available, so the
property that makes one array safe to update in place is shown here).

The scheme (the steps of the library's AA pattern, per fluid node x):
  odd step:  h_i = F[opp i][x - c_i]   if x - c_i is fluid, else F[i][x];
             f*_i -> F[i][x + c_i]     if x + c_i is fluid, else F[opp i][x];
  even step: h_i = F[i][x];  f*_i -> F[opp i][x].
Within one step every location must be read and written by a single node
only, and each node must write exactly the locations it read, so that no
ordering between threads matters."""
import itertools

import numpy as np
import pytest

import lbm_inputs as inp
import oracle


def _accesses(Q, tags, odd):
    c, _, opp = oracle.lattice(Q)
    nz, ny, nx = tags.shape
    fluid = tags <= oracle.FORCED
    owner = {}
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if not fluid[z, y, x]:
            continue
        reads, writes = set(), set()
        for i in range(Q):
            if odd:
                src = ((z - c[i][2]) % nz, (y - c[i][1]) % ny, (x - c[i][0]) % nx)
                dst = ((z + c[i][2]) % nz, (y + c[i][1]) % ny, (x + c[i][0]) % nx)
                reads.add((opp[i],) + src if fluid[src] else (i, z, y, x))
                writes.add((i,) + dst if fluid[dst] else (opp[i], z, y, x))
            else:
                reads.add((i, z, y, x))
                writes.add((opp[i], z, y, x))
        assert len(reads) == Q and reads == writes, (z, y, x)
        for loc in reads:
            assert loc not in owner, f"location {loc} touched by {owner.get(loc)} and {(z, y, x)}"
            owner[loc] = (z, y, x)
    return owner


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("seed", [1, 2])
def test_aa_steps_touch_each_location_once(Q, seed):
    shape = (4, 5, 6)
    tags = inp.random_tags(shape, seed=seed, p_solid=0.25, p_forced=0.3, p_wall=0.1, n_walls=2)
    for odd in (True, False):
        owner = _accesses(Q, tags, odd)
        n_fluid = int(np.sum(tags <= oracle.FORCED))
        assert len(owner) == Q * n_fluid  # a partition of the fluid nodes' Q slots


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 2, 3), (3, 1, 2)])
def test_aa_degenerate_rows_wrap_onto_the_node(shape):
    """Rows of one or two nodes: x - c_i and x + c_i wrap onto the node itself
    or onto one neighbour; the accesses still partition the slots."""
    tags = np.zeros(shape, np.uint8)
    for odd in (True, False):
        assert len(_accesses(19, tags, odd)) == 19 * int(np.prod(shape))
