"""Host logic of bench.py's roofline figures: algorithmic bytes per launch, kernel names, the flop
conventions and the lookup of ncu-measured DRAM traffic (no GPU)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

VH, NS = 16 * 16 * 16 * 32 // 2, 16


def test_hop_kernel_bytes():
    # K1 (FP32 hop + A^{-1}, store): 24 + 24 reals of 4 bytes per 5D half-site plus 8 links of 18 reals
    k1 = 100000 + 10000 + 1000
    assert bench.kernel_name(k1) == "k_hop<fp32,hop+A^-1,store>"
    assert bench.alg_bytes(k1, VH, NS) == VH * NS * 48 * 4 + VH * 8 * 18 * 4
    # K2A (FP32 hop + A own, CG_A): hopped field, own field, x and r read, x and r written
    k2a = 100000 + 10000 + 100 + 10 + 2
    assert bench.kernel_name(k2a) == "k_hop<fp32,hop+A*own,cg_a>"
    assert bench.alg_bytes(k2a, VH, NS) == VH * NS * 6 * 96 + VH * 8 * 18 * 4
    # FP16 storage: 2 bytes per real plus one 4-byte scale per field access
    k1h = 200000 + 10000 + 1000
    assert bench.alg_bytes(k1h, VH, NS) == VH * NS * 2 * (48 + 4) + VH * 8 * 18 * 4


def test_two_slice_kernel_names_and_bytes():
    # the two-slice kernels (storage digit + 5) read links as two rows: 8 x 12 reals per 4D half-site
    k1p = 600000 + 10000 + 1000
    assert bench.kernel_name(k1p) == "k_hop<two-slice,fp32,hop+A^-1,store>"
    assert bench.alg_bytes(k1p, VH, NS) == VH * NS * 48 * 4 + VH * 8 * 12 * 4
    # their bulk-copy form adds 1000000 to the key, like the bulk-staged kernels, with its own name
    assert bench.kernel_name(1000000 + k1p) == "k_hop<two-slice bulk,fp32,hop+A^-1,store>"
    assert bench.alg_bytes(1000000 + k1p, VH, NS) == bench.alg_bytes(k1p, VH, NS)
    assert bench.kernel_name(1000000 + 111000) == "k_hop<staged,fp32,hop+A^-1,store>"
    # FP16 two-slice: storage digit 7
    assert bench.kernel_name(700000 + 10000 + 100 + 10 + 3) == "k_hop<two-slice,fp16,hop+A*own,cg_b>"


def test_network_layer_bytes():
    # FP32 fields of 96 bytes per 5D half-site; BF16 intermediates are 48-byte rows per channel
    assert bench.alg_bytes(2000120, VH, NS) == VH * NS * (96 + 2 * 96) + VH * 8 * 18 * 4
    assert bench.alg_bytes(2001120, VH, NS) == VH * NS * (96 + 2 * 48) + VH * 8 * 18 * 4
    assert bench.alg_bytes(2000211, VH, NS) == VH * NS * (2 * 96 + 96 + 96) + VH * 8 * 18 * 4
    assert bench.alg_bytes(2001211, VH, NS) == VH * NS * (2 * 48 + 96 + 96) + VH * 8 * 18 * 4
    assert bench.kernel_name(2001211) == "k_net_layer<cin=2,cout=1,own,bf16>"
    assert bench.kernel_name(2000120) == "k_net_layer<cin=1,cout=2>"


def test_flop_conventions():
    assert bench.HOP_FLOPS == 8 * (12 + 2 * 66 + 24) - 24
    assert bench.CG_ITER_FLOPS == 4 * 1320 + 4 * 240 + 5 * 2 * 24 == 6480


def test_traffic_table_entries_name_measured_kernels():
    table = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    for e in table["entries"]:
        t = bench.dram_traffic(e["kernel"], tuple(e["dims"]), e["Ns"])
        assert t == e["dram_read_bytes"] + e["dram_write_bytes"] > 0
        # each entry names a kernel bench.py can report, and a summary that exists
        assert os.path.exists(os.path.join(ROOT, e["profile"]))
    assert bench.dram_traffic("k_hop<fp32,hop+A^-1,store>", (8, 8, 8, 8), 16) is None
    assert bench.dram_traffic("no such kernel", (16, 16, 16, 32), 16) is None


@pytest.mark.parametrize("key", [111000, 110112, 2001211, 4000100, 3000105])
def test_names_round_trip_to_known_kernels(key):
    assert bench.kernel_name(key).startswith("k_")
    assert bench.alg_bytes(key, VH, NS) >= 0


def test_average_plaquette():
    """bench.py's plaquette: 1 on unit links, gauge invariant, and equal to the oracle's on a seeded
    field (written independently there)."""
    import numpy as np
    from oracle import wilson
    from paper_1710_09621_gb300 import inputs
    dims = (4, 2, 2, 4)
    U1 = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, dims[3], dims[2], dims[1], dims[0], 3, 3)).copy()
    assert bench.average_plaquette(U1) == pytest.approx(1.0, abs=1e-15)
    U = inputs.random_su3_links(dims, 0.3, 7)
    p = bench.average_plaquette(U)
    assert p == pytest.approx(wilson.plaquette(U), abs=1e-14)
    assert 0.0 < p < 1.0
    # U_mu(x) -> G(x) U_mu(x) G(x + mu)^dag leaves it unchanged
    G = inputs.random_su3_links(dims, 1.0, 8)[0]
    axis = {0: 3, 1: 2, 2: 1, 3: 0}
    Ug = np.stack([G @ U[mu] @ np.roll(G, -1, axis=axis[mu]).conj().swapaxes(-1, -2) for mu in range(4)])
    assert bench.average_plaquette(Ug) == pytest.approx(p, abs=1e-13)
