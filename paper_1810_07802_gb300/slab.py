"""Domain decomposition of one y-periodic problem into y-slabs (bands of rows).

A band owns rows [r0, r1) of the problem and is stepped by an ordinary solver
on those rows plus HALO = 2 rows on each side: a periodic problem of
(r1 - r0) + 4 rows whose wrap-around reaches only its halo rows.  One step
of a cell reads psi-bar-plus of the rows next to it (the face
reconstruction, Eq. 27), and psi-bar-plus of such a row reads phi two rows
out (the gradient and Laplacian of Sec. II.B) and g and (phi u)^{n-1} on the
row itself; so before every step a band takes from each neighbour that
neighbour's two edge rows of every stored plane, and its own rows then get
the bits of the single-domain step.

The exchange is a pair of point-to-point messages per neighbour, no
collective: LocalExchange moves rows between bands held by one process
(one device), DistExchange between ranks over torch.distributed (NCCL
between GPUs; gloo on the CPU).  A band stepper is anything with
row_buffer(nrows), get_rows(row0, nrows, buf), set_rows(row0, nrows, buf),
step(n) and reduce_rows(row0, nrows): the GPU Solver of this package is one.

The FP64 reductions of the whole problem (phi mass, the steady-state
residuals of Eq. 44, max |u|) come from each band's sums over its own rows,
taken after a halo exchange: five sums added over the bands and one maximum
(an all-reduce of six numbers between ranks), then the ratios the
single-domain reduction forms.
"""
import numpy as np

HALO = 2


def bands(ny, world):
    """Rows [r0, r1) of each of `world` bands of a ny-row problem."""
    edges = np.linspace(0, ny, world + 1).round().astype(int)
    out = [(int(edges[r]), int(edges[r + 1])) for r in range(world)]
    if min(r1 - r0 for r0, r1 in out) < HALO:
        raise ValueError("each band needs at least %d rows" % HALO)
    return out


def band_problem(cfg, fields, r0, r1):
    """The band's own problem: rows r0 - HALO .. r1 + HALO - 1 (wrapped) of
    the periodic problem's parameters and initial fields."""
    if cfg.get("bc_y", "periodic") != "periodic":
        raise ValueError("the slab decomposition here is for y-periodic problems")
    ny = int(cfg["ny"])
    idx = np.arange(r0 - HALO, r1 + HALO) % ny
    bcfg = dict(cfg, ny=int(len(idx)))
    bfields = {k: (None if v is None else np.ascontiguousarray(np.asarray(v)[idx, :])) for k, v in fields.items()}
    return bcfg, bfields


class Band:
    """One band: a stepper on the band's problem and its halo bookkeeping.
    Own rows are HALO .. HALO + n_own - 1 of the stepper's grid."""

    def __init__(self, stepper, r0, r1):
        self.stepper, self.r0, self.r1 = stepper, r0, r1
        self.n_own = r1 - r0
        self.send_up = stepper.row_buffer(HALO)      # own top rows, for the band above
        self.send_down = stepper.row_buffer(HALO)    # own bottom rows, for the band below
        self.recv_below = stepper.row_buffer(HALO)   # the band below's top rows
        self.recv_above = stepper.row_buffer(HALO)   # the band above's bottom rows

    def pack(self):
        self.stepper.get_rows(HALO + self.n_own - HALO, HALO, self.send_up)
        self.stepper.get_rows(HALO, HALO, self.send_down)

    def unpack(self):
        self.stepper.set_rows(0, HALO, self.recv_below)
        self.stepper.set_rows(HALO + self.n_own, HALO, self.recv_above)

    def sums(self):
        """The band's reduction sums over its own rows (see combine)."""
        return self.stepper.reduce_rows(HALO, self.n_own)


def combine(sums, had_snapshot):
    """(phi mass, phi residual, u residual, max |u|) of the whole problem from
    the bands' summed sums [sum phi, sum phi^2, sum dphi^2, sum |u|^2,
    sum |du|^2] and the largest max |u|, as the single-domain reduction forms
    them (residuals 1.0 without a previous reduction)."""
    s = [float(x) for x in sums]
    if not had_snapshot:
        return s[0], 1.0, 1.0, s[5]
    rphi = s[2] / s[1] if s[1] > 0 else 0.0
    ru = s[4] / s[3] if s[3] > 0 else 0.0
    return s[0], rphi, ru, s[5]


def reduce_local(exchange, band_list):
    """The whole problem's reductions from bands held by one process.  The
    halo rows are refreshed first: u at a band's edge rows needs the
    gradient of phi across them."""
    exchange()
    parts = [b.sums() for b in band_list]
    tot = np.zeros(6)
    for v, _ in parts:
        tot[:5] += v[:5]
        tot[5] = max(tot[5], v[5])
    return combine(tot, all(h for _, h in parts))


class LocalExchange:
    """Halo exchange between the bands of one process, in ring order (band b's
    upper neighbour is band b + 1, periodically)."""

    def __init__(self, band_list):
        self.bands = band_list

    def __call__(self):
        n = len(self.bands)
        for b in self.bands:
            b.pack()
        for i, b in enumerate(self.bands):
            up, down = self.bands[(i + 1) % n], self.bands[(i - 1) % n]
            up.recv_below.copy_(b.send_up)
            down.recv_above.copy_(b.send_down)
        for b in self.bands:
            b.unpack()


class DistExchange:
    """Halo exchange of this rank's band with its neighbours over
    torch.distributed: sends to the rank above and below, then receives from
    below and above, posted in that order in one batch (so that with two
    ranks, where both neighbours are one rank, the messages pair up by order;
    the tags do the same where the backend honours them)."""

    def __init__(self, band, rank, world, group=None):
        self.band, self.rank, self.world, self.group = band, rank, world, group

    def __call__(self):
        import torch.distributed as dist

        b = self.band
        b.pack()
        up, down = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        ops = [dist.P2POp(dist.isend, b.send_up, up, self.group, 0),
               dist.P2POp(dist.isend, b.send_down, down, self.group, 1),
               dist.P2POp(dist.irecv, b.recv_below, down, self.group, 0),
               dist.P2POp(dist.irecv, b.recv_above, up, self.group, 1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        b.unpack()

    def reduce(self):
        """The whole problem's reductions: this rank's band sums, all-reduced
        (a sum of five, a maximum of one) over the ranks, after a halo
        exchange (u at the band's edge rows needs phi across them)."""
        import torch
        import torch.distributed as dist

        self()
        v, had = self.band.sums()
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor(list(v[:5]) + [1.0 if had else 0.0], dtype=torch.float64, device=dev)
        m = torch.tensor([v[5]], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        dist.all_reduce(m, op=dist.ReduceOp.MAX, group=self.group)
        t, m = t.cpu().numpy(), m.cpu().numpy()
        return combine(list(t[:5]) + [m[0]], t[5] == self.world)


def step_bands(exchange, band_list, n):
    """n steps of every band: exchange the halos, then one step of each band."""
    for _ in range(int(n)):
        exchange()
        for b in band_list:
            b.stepper.step(1)
