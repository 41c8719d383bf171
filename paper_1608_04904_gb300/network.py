"""Host-side preparation of a bead network held by iterative RATTLE (the
paper's Janus integrator, §1.4): an edge colouring of the links.

Links of one colour share no bead, so one sweep of the iterative RATTLE can
correct all links of a colour at the same time -- one thread per link -- and
give exactly what correcting them one after another gives.  A sweep colour
by colour is therefore the sequential sweep over the links listed colour by
colour (`order_by_color`), which is the order a parallel kernel reproduces
bit for bit."""
from __future__ import annotations

import numpy as np


def color_links(links, n_beads: int) -> np.ndarray:
    """Greedy edge colouring: every link gets the smallest colour not yet used
    by a link at either of its beads.  Uses at most 2 d - 1 colours for a
    largest bead degree d.  Returns one colour per link."""
    used = [set() for _ in range(int(n_beads))]
    colors = np.empty(len(links), dtype=np.int32)
    for k, (a, b) in enumerate(links):
        if a == b or not (0 <= a < n_beads and 0 <= b < n_beads):
            raise ValueError(f"link {k} ({a}, {b}) is not a pair of distinct beads")
        c = 0
        while c in used[a] or c in used[b]:
            c += 1
        colors[k] = c
        used[a].add(c)
        used[b].add(c)
    return colors


def order_by_color(links, colors) -> np.ndarray:
    """Link indices colour by colour (stable within a colour): the sequential
    order equivalent to a colour-by-colour parallel sweep."""
    return np.argsort(np.asarray(colors), kind="stable")
