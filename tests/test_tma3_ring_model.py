"""CPU model of the 3-D TMA two-sweep kernel's plane rings (k_jacobi3_x2t in
paper_1108_2045_gb300/csrc/homg_kernels.cu), run without a GPU.

A block marches first-sweep planes zf = z0 - 1 .. zl (zl = min(z0 + RZ, n)) and second-sweep planes
zs = zf - 1. With prefetch distance D, the input iterate's planes live in a ring of D + 3 slots
(slot (p + 2) mod (D + 3)), the source's in D + 2 slots (slot (p + 1) mod (D + 2)), the first
sweep's in 3 slots (slot (p + 1) mod 3). Step s needs iterate planes s - 1 .. s + 1 and source plane
s. Set-up copies iterate planes z0 - 2 .. z0 and source plane z0 - 1 (step z0 - 1's data) on barrier
D + 1, then for the steps s = z0 .. z0 + D - 2 their iterate plane s + 1 and source plane s on
barrier s mod (D + 1). Step zf first copies step zf + D's planes (iterate zf + D + 1, source zf + D,
while zf + D <= zl) on barrier (zf + D) mod (D + 1), then waits for its own (barrier D + 1 on the
first step, zf mod (D + 1) after). The model replays that schedule and checks that every read finds
the plane it expects, that no copy lands in a slot still to be read in the step, and that every
barrier phase waited on was armed exactly once.
"""

import pytest


def replay(z0, RZ, n, D, e_slots=None, g_slots=None, s_slots=3):
    e_slots = e_slots or D + 3
    g_slots = g_slots or D + 2
    NB = D + 1
    E, G, S = [None] * e_slots, [None] * g_slots, [None] * s_slots
    armed, arm_ph, wait_ph, waits = {}, {}, {}, []
    zl = min(z0 + RZ, n)
    zout = min(z0 + RZ - 1, n - 1)

    def slot(kind, p):
        if kind == "E":
            return (p + 2) % e_slots
        if kind == "G":
            return (p + 1) % g_slots
        return (p + 1) % s_slots

    reading = set()

    def put(kind, ring, p):
        k = slot(kind, p)
        assert (kind, k) not in reading, ("write into a slot being read", kind, p)
        ring[k] = p

    def get(kind, ring, p):
        k = slot(kind, p)
        assert ring[k] == p, ("slot holds another plane", kind, p, ring[k])
        reading.add((kind, k))

    def arm(bar, what):
        ph = arm_ph.get(bar, 0)
        armed[(bar, ph)] = what
        arm_ph[bar] = ph + 1

    def wait(bar):
        ph = wait_ph.get(bar, 0)
        assert (bar, ph) in armed, ("wait on an unarmed phase", bar, ph)
        wait_ph[bar] = ph + 1
        waits.append((bar, ph))

    # set-up: step z0 - 1's planes, then steps z0 .. z0 + D - 2
    for p in (z0 - 2, z0 - 1, z0):
        put("E", E, p)
    put("G", G, z0 - 1)
    arm(NB, "init")
    for st in range(z0, min(z0 + D - 1, zl + 1)):
        put("E", E, st + 1)
        put("G", G, st)
        arm(st % NB, st)
    for zf in range(z0 - 1, zl + 1):
        reading.clear()
        if zf + D <= zl:  # copies for step zf + D
            put("E", E, zf + D + 1)
            put("G", G, zf + D)
            arm((zf + D) % NB, zf + D)
        wait(NB if zf == z0 - 1 else zf % NB)
        for p in (zf - 1, zf, zf + 1):  # first sweep at zf
            get("E", E, p)
        get("G", G, zf)
        put("S", S, zf)
        reading.clear()  # block barrier
        zs = zf - 1
        if z0 <= zs <= zout:  # second sweep at zs
            for p in (zs - 1, zs, zs + 1):
                get("S", S, p)
            get("G", G, zs)
        reading.clear()  # block barrier
    assert set(armed) == set(waits)


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("z0,RZ,n", [(1, 32, 512), (33, 32, 512), (481, 32, 512), (1, 8, 8), (1, 1, 4),
                                     (5, 4, 16), (1, 16, 2), (9, 16, 16), (1, 32, 256), (225, 32, 256)])
def test_plane_ring_schedule(z0, RZ, n, D):
    replay(z0, RZ, n, D)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_model_catches_short_rings(D):
    with pytest.raises(AssertionError):
        replay(1, 32, 512, D, e_slots=D + 2)
    with pytest.raises(AssertionError):
        replay(1, 32, 512, D, g_slots=D + 1)
    with pytest.raises(AssertionError):
        replay(1, 32, 512, D, s_slots=2)
