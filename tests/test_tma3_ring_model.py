"""CPU model of the 3-D TMA two-sweep kernel's plane rings (k_jacobi3_x2t in
paper_1108_2045_gb300/csrc/homg_kernels.cu), run without a GPU.

A block marches first-sweep planes zf = z0 - 1 .. z0 + RZ and second-sweep planes zs = zf - 1. The
input iterate's planes live in a ring of 4 slots (slot (p + 2) mod 4), the source's in 3 slots
(slot (p + 1) mod 3), the first sweep's in 3 slots (slot (p + 1) mod 3). Set-up copies iterate
planes z0 - 2 .. z0 and source plane z0 - 1 on barrier INIT; step zf copies iterate plane zf + 2 and
source plane zf + 1 on barrier LB[(zf + 4) mod 4] (while they are needed) and waits for the copies
issued one step earlier. The model replays the schedule and checks that every read finds the plane
it expects, that no copy or store lands in a slot still to be read, and that every barrier phase
waited on was armed exactly once.
"""

import pytest


def replay(z0, RZ, n, e_slots=4, g_slots=3, s_slots=3):
    E, G, S = [None] * e_slots, [None] * g_slots, [None] * s_slots
    armed = {}    # (barrier, phase) -> planes it carries
    phase = {}    # barrier -> next phase to arm / wait
    waits = []
    zlast = z0 + RZ  # last first-sweep plane

    def arm(bar, planes):
        ph = phase.get(("arm", bar), 0)
        assert (bar, ph) not in armed
        armed[(bar, ph)] = planes
        phase[("arm", bar)] = ph + 1

    def wait(bar):
        ph = phase.get(("wait", bar), 0)
        assert (bar, ph) in armed, ("wait on an unarmed phase", bar, ph)
        phase[("wait", bar)] = ph + 1
        waits.append((bar, ph))
        return armed[(bar, ph)]

    reading = set()  # slots read in the current phase of a step: ("E", k) ...

    def put(kind, ring, slots, p):
        k = (p + 2) % slots if kind == "E" else (p + 1) % slots
        assert (kind, k) not in reading, ("write into a slot being read", kind, p)
        ring[k] = p

    def get(kind, ring, slots, p):
        k = (p + 2) % slots if kind == "E" else (p + 1) % slots
        assert ring[k] == p, ("slot holds another plane", kind, p, ring[k])
        reading.add((kind, k))

    # set-up copies
    for p in (z0 - 2, z0 - 1, z0):
        put("E", E, e_slots, p)
    put("G", G, g_slots, z0 - 1)
    arm("INIT", ("E", z0 - 2, z0 - 1, z0, "G", z0 - 1))
    for zf in range(z0 - 1, zlast + 1):
        # (a) copies for the next step, into slots freed by the previous step's barriers
        if zf + 2 <= zlast + 1:
            put("E", E, e_slots, zf + 2)
            if zf + 1 <= zlast:
                put("G", G, g_slots, zf + 1)
            arm((zf + 4) % 4, ("E", zf + 2))
        # (b) the data this step needs
        wait("INIT" if zf == z0 - 1 else (zf + 3) % 4)
        # (c) first sweep at zf
        reading.clear()
        for p in (zf - 1, zf, zf + 1):
            get("E", E, e_slots, p)
        get("G", G, g_slots, zf)
        put("S", S, s_slots, zf)
        reading.clear()  # (d) block barrier
        # (e) second sweep at zs = zf - 1
        zs = zf - 1
        if z0 <= zs <= min(z0 + RZ - 1, n - 1):
            for p in (zs - 1, zs, zs + 1):
                get("S", S, s_slots, p)
            get("G", G, g_slots, zs)
        reading.clear()  # (f) block barrier
    # every armed phase was waited on, or is a copy that was issued past the last step (none)
    assert set(armed) == set(waits)


@pytest.mark.parametrize("z0,RZ,n", [(1, 32, 512), (33, 32, 512), (481, 32, 512), (1, 8, 8), (1, 1, 4),
                                     (5, 4, 16), (1, 16, 2), (9, 16, 16)])
def test_plane_ring_schedule(z0, RZ, n):
    replay(z0, RZ, n)


def test_model_catches_short_rings():
    with pytest.raises(AssertionError):
        replay(1, 32, 512, e_slots=3)
    with pytest.raises(AssertionError):
        replay(1, 32, 512, s_slots=2)
