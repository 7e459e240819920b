"""Domain decomposition of one problem into y-slabs (bands of rows).

A band owns rows [r0, r1) of the problem and is stepped by an ordinary solver
on those rows plus `halo` rows on each side that has a neighbouring band.  One
step of a cell reads psi-bar-plus of the rows next to it (the face
reconstruction, Eq. 27), and psi-bar-plus of such a row reads phi one row
further out (the gradient and Laplacian of Sec. II.B) and g and
(phi u)^{n-1} on the row itself: two halo rows.  The upwind reconstruction
reads the profile of the cell a direction leaves, one row further again:
three halo rows.  Before every step a band takes from each neighbour that
neighbour's `halo` edge rows of every stored plane, and its own rows then get
the bits of the single-domain step.

Boundaries.  A y-periodic problem is cut into bands that are periodic
problems of their own rows plus a halo on both sides; the wrap-around of a
band's grid reaches only its halo rows.  A problem with no-slip walls in y is
cut into bands that are walled problems: the first band has no halo below
(its wall is the problem's), the last none above, and the walls a band's
grid has at an inner edge touch only its outermost halo row (the phi
mirror of the stencils, the one-sided y-slopes of that row's x-faces and
the wall face itself), which its own rows never read.  Prescribed velocity
fields that depend on position are not decomposed.

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

HALO = 2          # halo rows of the central reconstruction
HALO_UPWIND = 3   # halo rows of the upwind reconstruction


def halo_rows(cfg):
    """Halo rows a band of this problem needs on each side with a neighbour."""
    return HALO_UPWIND if cfg.get("recon", "central") == "upwind" else HALO


def _walled(cfg):
    bc = cfg.get("bc_y", "periodic")
    if bc not in ("periodic", "wall"):
        raise ValueError("unknown y-boundary %r" % (bc,))
    return bc == "wall"


def bands(ny, world, halo=HALO):
    """Rows [r0, r1) of each of `world` bands of a ny-row problem (each band
    at least `halo` rows, so that its edge rows fill a neighbour's halo)."""
    edges = np.linspace(0, ny, world + 1).round().astype(int)
    out = [(int(edges[r]), int(edges[r + 1])) for r in range(world)]
    if min(r1 - r0 for r0, r1 in out) < halo:
        raise ValueError("each band needs at least %d rows" % halo)
    return out


def band_layout(cfg, r0, r1, halo=None):
    """(halo, lo, hi): the halo width and the halo rows of band [r0, r1)
    below and above its own rows (0 at a wall of the problem)."""
    h = halo_rows(cfg) if halo is None else int(halo)
    ny = int(cfg["ny"])
    if not 0 <= r0 < r1 <= ny:
        raise ValueError("rows [%d, %d) are not inside the problem" % (r0, r1))
    walled = _walled(cfg)
    lo = 0 if (walled and r0 == 0) else h
    hi = 0 if (walled and r1 == ny) else h
    return h, lo, hi


def band_problem(cfg, fields, r0, r1, halo=None):
    """The band's own problem: its rows and halo rows (wrapped if periodic)
    of the problem's parameters and initial fields."""
    model = cfg.get("model", "coupled")
    vel = cfg.get("velocity_field", "uniform")
    if model != "coupled" and vel not in ("uniform", 0, None):
        raise ValueError("prescribed velocity fields that depend on position are not decomposed")
    h, lo, hi = band_layout(cfg, r0, r1, halo)
    ny = int(cfg["ny"])
    idx = np.arange(r0 - lo, r1 + hi) % ny
    bcfg = dict(cfg, ny=int(len(idx)))
    bfields = {k: (None if v is None else np.ascontiguousarray(np.asarray(v)[idx, :])) for k, v in fields.items()}
    return bcfg, bfields


class Band:
    """One band: a stepper on the band's problem (band_problem) and its halo
    bookkeeping.  Own rows are lo .. lo + n_own - 1 of the stepper's grid;
    cfg is the whole problem's (for the halo width and the boundaries)."""

    def __init__(self, stepper, r0, r1, cfg=None, halo=None):
        self.stepper, self.r0, self.r1 = stepper, r0, r1
        self.n_own = r1 - r0
        if cfg is None:   # a periodic problem, central reconstruction
            h = HALO if halo is None else int(halo)
            self.halo, self.lo, self.hi = h, h, h
        else:
            self.halo, self.lo, self.hi = band_layout(cfg, r0, r1, halo)
        if self.n_own < self.halo:
            raise ValueError("a band needs at least %d own rows" % self.halo)
        self.own = slice(self.lo, self.lo + self.n_own)
        h = self.halo
        # own top rows for the band above, own bottom rows for the band below,
        # and the rows received from below and above
        self.send_up = stepper.row_buffer(h) if self.hi else None
        self.send_down = stepper.row_buffer(h) if self.lo else None
        self.recv_below = stepper.row_buffer(h) if self.lo else None
        self.recv_above = stepper.row_buffer(h) if self.hi else None

    def pack(self):
        if self.hi:
            self.stepper.get_rows(self.lo + self.n_own - self.halo, self.halo, self.send_up)
        if self.lo:
            self.stepper.get_rows(self.lo, self.halo, self.send_down)

    def unpack(self):
        if self.lo:
            self.stepper.set_rows(0, self.halo, self.recv_below)
        if self.hi:
            self.stepper.set_rows(self.lo + self.n_own, self.halo, self.recv_above)

    def sums(self):
        """The band's reduction sums over its own rows (see combine)."""
        return self.stepper.reduce_rows(self.lo, self.n_own)


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
    """Halo exchange between the bands of one process, listed bottom to top
    (band b's upper neighbour is band b + 1, periodically unless the bands are
    walled at the ends)."""

    def __init__(self, band_list):
        self.bands = band_list

    def __call__(self):
        n = len(self.bands)
        for b in self.bands:
            b.pack()
        for i, b in enumerate(self.bands):
            if b.hi:
                self.bands[(i + 1) % n].recv_below.copy_(b.send_up)
            if b.lo:
                self.bands[(i - 1) % n].recv_above.copy_(b.send_down)
        for b in self.bands:
            b.unpack()


class DistExchange:
    """Halo exchange of this rank's band with its neighbours over
    torch.distributed (rank r holds the r-th band from the bottom): sends to
    the rank above and below, then receives from below and above, posted in
    that order in one batch (so that with two periodic ranks, where both
    neighbours are one rank, the messages pair up by order; the tags do the
    same where the backend honours them).  A band at a wall of the problem
    has no neighbour on that side; a single rank's periodic band is its own
    neighbour, and its rows are copied in place."""

    def __init__(self, band, rank, world, group=None):
        self.band, self.rank, self.world, self.group = band, rank, world, group

    def __call__(self):
        import torch.distributed as dist

        b = self.band
        b.pack()
        if self.world == 1:   # a periodic problem on one rank: its own edge rows wrap around
            if b.lo:
                b.recv_below.copy_(b.send_up)
                b.recv_above.copy_(b.send_down)
            b.unpack()
            return
        up, down = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        ops = []
        if b.hi:
            ops.append(dist.P2POp(dist.isend, b.send_up, up, self.group, 0))
        if b.lo:
            ops.append(dist.P2POp(dist.isend, b.send_down, down, self.group, 1))
            ops.append(dist.P2POp(dist.irecv, b.recv_below, down, self.group, 0))
        if b.hi:
            ops.append(dist.P2POp(dist.irecv, b.recv_above, up, self.group, 1))
        if ops:
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
