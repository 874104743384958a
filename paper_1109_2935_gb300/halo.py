"""Host side of the domain decomposition (Sec. 6) across processes, one rank per GPU:
face exchange with the neighbours in every cut dimension and global sums, each bounded
by a deadline. The faces are whatever the caller packs (the library packs spin-projected
boundary slices, 12 reals per face site); this module only moves them. A message that
does not arrive in time raises HaloTimeout (code ERR_TIMEOUT = -8, as in the C ABI)
instead of blocking: a rank that died or stopped sending is reported to the caller,
which then tears the process group down (after a timeout the backend may have closed
the connection, so no further collective is attempted on that group).

The ranks form a grid (g_x, g_y, g_z, g_t) (default (1, 1, 1, P): t-slabs), rank index
c_x + g_x (c_y + g_y (c_z + g_z c_t)). In dimension mu a rank's next rank is c_mu + 1
(mod g_mu), its previous rank c_mu - 1. Each exchange in mu sends the rank's first
mu-slice to the previous rank (which uses it for its forward mu-hops) and its last slice
to the next rank (backward mu-hops). In a dimension with one rank the faces are its own
(periodic wrap), copied without messages."""
import datetime
import time

import torch
import torch.distributed as dist

ERR_TIMEOUT = -8
TAG_TO_PREV, TAG_TO_NEXT = 101, 102


class HaloTimeout(RuntimeError):
    def __init__(self, what, seconds):
        super().__init__(f"ERR_TIMEOUT: {what} not complete after {seconds:.3f} s")
        self.code = ERR_TIMEOUT


class HaloExchange:
    def __init__(self, timeout_s=1.0, group=None, grid=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.grid = tuple(grid) if grid is not None else (1, 1, 1, self.world)
        if len(self.grid) != 4 or any(g < 1 for g in self.grid) or \
                self.grid[0] * self.grid[1] * self.grid[2] * self.grid[3] != self.world:
            raise ValueError(f"rank grid {self.grid} does not match {self.world} ranks")
        r, co = self.rank, []
        for g in self.grid:
            co.append(r % g)
            r //= g
        self.coords = tuple(co)
        self.next = tuple(self._rank_at(mu, +1) for mu in range(4))
        self.prev = tuple(self._rank_at(mu, -1) for mu in range(4))
        self.timeout_s = timeout_s

    def _rank_at(self, mu, step):
        co = list(self.coords)
        co[mu] = (co[mu] + step) % self.grid[mu]
        gx, gy, gz, _ = self.grid
        return co[0] + gx * (co[1] + gy * (co[2] + gz * co[3]))

    def _wait(self, works, what):
        deadline = time.monotonic() + self.timeout_s
        for w in works:
            left = deadline - time.monotonic()
            if left <= 0:
                raise HaloTimeout(what, self.timeout_s)
            try:
                done = w.wait(timeout=datetime.timedelta(seconds=left))
            except RuntimeError as e:  # the backend reports its own timeout as an error
                if "timed out" in str(e).lower() or "timeout" in str(e).lower():
                    raise HaloTimeout(what, self.timeout_s) from e
                raise
            if done is False:
                raise HaloTimeout(what, self.timeout_s)

    def exchange(self, to_prev, to_next, mu=3):
        """Send `to_prev` (first mu-slice) to the previous rank in mu and `to_next` (last
        slice) to the next rank; return (from_next, from_prev): the next rank's first slice
        and the previous rank's last slice."""
        if self.grid[mu] == 1:
            return to_prev.clone(), to_next.clone()
        from_next = torch.empty_like(to_prev)
        from_prev = torch.empty_like(to_next)
        tp, tn = TAG_TO_PREV + 10 * mu, TAG_TO_NEXT + 10 * mu
        works = [dist.irecv(from_next, src=self.next[mu], tag=tp, group=self.group),
                 dist.irecv(from_prev, src=self.prev[mu], tag=tn, group=self.group),
                 dist.isend(to_prev.contiguous(), dst=self.prev[mu], tag=tp, group=self.group),
                 dist.isend(to_next.contiguous(), dst=self.next[mu], tag=tn, group=self.group)]
        self._wait(works, f"halo exchange in dimension {mu}")
        return from_next, from_prev

    def allreduce(self, x):
        """Sum of x over the ranks, in place."""
        if self.world > 1:
            self._wait([dist.all_reduce(x, group=self.group, async_op=True)], "allreduce")
        return x
