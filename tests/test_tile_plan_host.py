"""Host check of the tile-staged stencil's copy plan (WD_STENCIL_TILE,
csrc/dslash_tt.cuh) against the lattice's neighbour table (Section 3.1: the
Wilson hop couples x to x +- mu; even-odd site numbering cb = lex / 2).

The test restates, in Python, what the producer warp issues for one stage
(tile, direction) -- the runs of consecutive neighbour rows, one bulk copy per
spinor component and link row per run, spread over the warp's lanes -- and the
index every consumer thread reads from the stage.  For every tile and
direction of the lattices below (both parities, FP32 and 16-bit spinor
layouts) it checks that the copies stay inside the fields and the stage, fill
each stage slot exactly once, and that each consumer reads the neighbour
spinor and link the hop needs.  No GPU is used.
"""
import pytest

TILE = 512          # TT_TILE: output sites per tile


def _cb_of(L, c):
    Lx, Ly, Lz, Lt = L
    return ((((c[3] * Lz + c[2]) * Ly + c[1]) * Lx + c[0]) >> 1)


def _ffs(m):
    return (m & -m).bit_length() if m else 0


def _eligible(L):
    Lh, Vh = L[0] // 2, L[0] * L[1] * L[2] * L[3] // 2
    return Lh >= 8 and Lh % 4 == 0 and TILE % Lh == 0 and TILE // Lh <= 32 and Vh % TILE == 0


def _check(L, par, ncopy):
    Lx, Ly, Lz, Lt = L
    Lh, Vh = Lx // 2, Lx * Ly * Lz * Lt // 2
    nr = TILE // Lh
    for tile in range(Vh // TILE):
        R0 = tile * nr
        lanes = []
        for lane in range(32):
            R = R0 + (lane if lane < nr else 0)
            lanes.append((R, R % Ly, (R // Ly) % Lz, (R // Ly) // Lz))
        for D in range(8):
            mu, fwd = D >> 1, (D & 1) == 0
            Rn = []
            for R, y, z, t in lanes:            # neighbour row of each lane's row
                if mu == 0:
                    Rn.append(R)
                elif mu == 1:
                    Rn.append(R + ((1 - Ly if y + 1 == Ly else 1) if fwd else (Ly - 1 if y == 0 else -1)))
                elif mu == 2:
                    Rn.append(R + Ly * ((1 - Lz if z + 1 == Lz else 1) if fwd else (Lz - 1 if z == 0 else -1)))
                else:
                    Rn.append(R + Ly * Lz * ((1 - Lt if t + 1 == Lt else 1) if fwd else (Lt - 1 if t == 0 else -1)))
            starts = 0
            for lane in range(nr):
                if lane == 0 or Rn[lane] != Rn[lane - 1] + 1:
                    starts |= 1 << lane
            npc = bin(starts).count("1")
            per = ncopy if fwd else ncopy + 3
            ntup = npc * per + (3 if fwd else 0)
            spin = [[None] * TILE for _ in range(ncopy)]
            link = [[None] * TILE for _ in range(3)]
            for k0 in range(0, ntup, 32):
                for lane in range(32):
                    k = k0 + lane
                    p, j = divmod(k, per)
                    if k >= npc * per:
                        p = 0
                    m = starts
                    for _ in range(p):
                        m &= m - 1
                    r0 = _ffs(m) - 1
                    later = m & (m - 1)
                    r1 = _ffs(later) - 1 if later else nr
                    if k < npc * per:
                        dsite, n, src = r0 * Lh, (r1 - r0) * Lh, Rn[r0] * Lh
                        assert 0 <= src and src + n <= Vh and dsite + n <= TILE and n > 0
                        tgt = spin[j] if j < ncopy else link[j - ncopy]
                        for a in range(n):
                            assert tgt[dsite + a] is None
                            tgt[dsite + a] = ("b" if j >= ncopy else "s", src + a)
                    elif k < ntup:
                        for a in range(TILE):
                            assert link[k - npc * per][a] is None
                            link[k - npc * per][a] = ("f", R0 * Lh + a)
            assert all(v is not None for arr in spin + link for v in arr)
            for i in range(TILE):                # what every consumer thread reads
                cb = tile * TILE + i
                ir, xh = divmod(i, Lh)
                R = tile * nr + ir
                y, z, t = R % Ly, (R // Ly) % Lz, (R // Ly) // Lz
                x = 2 * xh + ((par + y + z + t) & 1)
                xodd = (x & 1) == 1
                ixf = ir * Lh + ((0 if xh + 1 == Lh else xh + 1) if xodd else xh)
                ixb = ir * Lh + (xh if xodd else (Lh - 1 if xh == 0 else xh - 1))
                is_ = (ixf if fwd else ixb) if mu == 0 else i
                il = i if fwd else is_
                nbc = [x, y, z, t]
                nbc[mu] = (nbc[mu] + 1) % L[mu] if fwd else (nbc[mu] - 1) % L[mu]
                want = _cb_of(L, nbc)
                for j in range(ncopy):
                    assert spin[j][is_] == ("s", want)
                for j in range(3):
                    assert link[j][il] == (("f", cb) if fwd else ("b", want))


@pytest.mark.parametrize("dims", [(32, 2, 2, 16), (32, 4, 6, 8), (64, 2, 4, 8), (32, 8, 2, 8)],
                         ids=lambda d: "x".join(map(str, d)))
def test_tile_copy_plan_covers_the_neighbour_table(dims):
    assert _eligible(dims)
    for par in (0, 1):
        for ncopy in (6, 4):                     # FP32 spinors; 16-bit words + norms
            _check(dims, par, ncopy)


def test_ineligible_lattices_are_excluded():
    # rows of fewer than 8 sites, more than 32 rows per tile, or a partial tile
    for dims in [(8, 8, 8, 16), (12, 12, 12, 24), (16, 8, 6, 10), (4, 4, 4, 4)]:
        assert not _eligible(dims)
