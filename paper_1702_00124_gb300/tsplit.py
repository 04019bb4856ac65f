"""Time-direction domain decomposition of one lattice over several GPUs: the
exchange plan and the global sums (Section 2: the solver of K needs a global
inner product per iteration; Section 3.1: the nearest-neighbour Wilson stencil).

Not on the single-GPU path, which runs one lattice per GPU.  The lattice
Lx x Ly x Lz x Lt is cut into `world` slabs of Lt / world time slices; rank r
holds slices [r nt, (r + 1) nt) of every field.  Only the hops in t cross a
cut.  Per hop D_{p <- 1-p} rank r
  - receives from rank r+1 the forward face: for each site of parity 1-p on
    that rank's first slice, the half spinor h = upper spins of (1 -+ g_t) psi
    (12 reals; the lower spins are -+h in the chiral basis), which rank r
    multiplies by its own U_t of its last slice;
  - receives from rank r-1 the backward face: for each site of parity 1-p on
    that rank's last slice, U_t(x)^dag applied to the upper spins of
    (1 +- g_t) psi(x) (12 reals), computed there because the link lives there;
  - applies the antiperiodic sign -1 to a face that crosses t = Lt-1 -> 0.
So a hop moves 2 x (Lx Ly Lz / 2) x 12 reals per rank and direction pair, the
links never move (the T step is local), and every CG dot product or norm is
one FP64 all-reduce of the ranks' partial sums.  The exchange uses
torch.distributed point-to-point calls (NCCL between GPUs, gloo on the CPU).
"""


def slab(lt, rank, world):
    """First global time slice and slice count of rank's slab."""
    # an even slice count keeps every slab's first slice even, so local and
    # global site parities agree
    if world < 1 or lt % world != 0 or (lt // world) % 2 != 0:
        raise ValueError("Lt must split into equal slabs of an even number of slices")
    nt = lt // world
    return rank * nt, nt


def neighbours(rank, world):
    """(rank holding the next slices, rank holding the previous slices), periodic."""
    return (rank + 1) % world, (rank - 1) % world


def face_sites(dims):
    """Sites of one parity on one time slice: the length of a face."""
    lx, ly, lz, _ = dims
    return lx * ly * lz // 2


def face_bytes(dims, bytes_per_real):
    """Bytes one rank sends per hop: two faces of 12-real half spinors."""
    return 2 * face_sites(dims) * 12 * bytes_per_real


def crosses_boundary(rank, world, forward):
    """Whether the face a rank receives crosses the antiperiodic cut t = Lt-1 -> 0."""
    return (rank == world - 1) if forward else (rank == 0)


def exchange_faces(dist, rank, world, to_prev, to_next, from_next, from_prev):
    """Send `to_prev` (this rank's forward face, for rank-1) and `to_next` (its
    backward face, for rank+1); receive into `from_next` and `from_prev`.
    Tensors of equal shape; one isend / irecv pair per direction."""
    nxt, prv = neighbours(rank, world)
    reqs = [dist.isend(to_prev, prv), dist.isend(to_next, nxt),
            dist.irecv(from_next, nxt), dist.irecv(from_prev, prv)]
    for r in reqs:
        r.wait()


def global_sum(dist, value, device="cpu"):
    """FP64 sum of the ranks' partial sums (a CG dot product or norm)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
