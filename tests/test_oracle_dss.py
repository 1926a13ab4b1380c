"""Pins of the oracle's DSS forward pass (Section III-B, Eqs. 18-22; Table 2)."""
import os

import numpy as np
import pytest

import synth
from oracle import dss, fem, partition as pt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [line.split() for line in fh if line.strip() and not line.startswith("#")]


def test_weight_count_reproduces_table2():
    rows = _rows("table2_nb_weights.txt")
    assert len(rows) == 10
    for kbar, d, count in rows:
        assert dss.n_weights(int(kbar), int(d)) == int(count)
        assert synth.n_weights_per_block(int(d)) * int(kbar) == int(count)


def _two_node_weights():
    def block(psi_b2, dec):
        return np.concatenate([
            [1, 2, 3, 4, 5], [0.5], [2], [0.25],          # phi_out
            [-1, 1, 2, -3, 1], [0.0], [-1], [0.5],        # phi_in
            [1, 1, 0.5, -0.5], [0.0], [3], [psi_b2],      # psi
            dec,                                          # decoder W1 b1 W2 b2
        ])
    return np.concatenate([block(-1.0, [2, -1, 4, 0.5]), block(0.0, [1, 0, 1, 0])])


def test_two_node_hand_example():
    xy = np.array([[0.0, 0.0], [1.0, 0.0]])
    src, dst = np.array([1]), np.array([0])
    w = _two_node_weights()
    expected = {int(k): float(v) for k, v in _rows("dss_two_node.txt")}
    got1 = dss.forward(xy, 1, src, dst, np.array([1.0]), w[:w.size // 2], 1, 1, 0.5, 1.0)
    got2 = dss.forward(xy, 1, src, dst, np.array([1.0]), w, 2, 1, 0.5, 1.0)
    assert got1[0] == expected[1]
    assert got2[0] == expected[2]


@pytest.fixture(scope="module")
def graph():
    m = synth.square_mesh(15, seed=2)
    P = fem.assemble(m.xy, m.tri, coeffs=synth.poly_coeffs(2))
    D = pt.decompose(P, 2, 1)
    g = pt.local_graph(P, D.sets[0])
    hbar = pt.mean_edge_length(m.xy, m.tri)
    c = synth.residual_vector(g.n_int, 7)
    return g, c / np.linalg.norm(c), hbar


KB, DD = 4, 6


def test_alpha_zero_gives_decoder_of_zero_state(graph):
    g, c, hbar = graph
    w = synth.dss_weights(KB, DD, 3, bias_scale=0.5)
    out = dss.forward(g.xy, g.n_int, g.src, g.dst, c, w, KB, DD, 0.0, hbar)
    last = dss.unpack(w, KB, DD)[-1]
    value = last["dec.W2"] @ np.maximum(last["dec.b1"], 0.0) + last["dec.b2"]
    assert np.allclose(out, value[0], rtol=0, atol=1e-15)


def test_factorised_form_agrees(graph):
    g, c, hbar = graph
    w = synth.dss_weights(KB, DD, 4, bias_scale=0.3)
    a = dss.forward(g.xy, g.n_int, g.src, g.dst, c, w, KB, DD, 0.2, hbar)
    b = dss.forward_factorised(g.xy, g.n_int, g.src, g.dst, c, w, KB, DD, 0.2, hbar)
    assert np.max(np.abs(a - b)) < 1e-13 * max(1.0, np.max(np.abs(a)))


def test_permutation_equivariance_and_translation_invariance(graph):
    g, c, hbar = graph
    w = synth.dss_weights(KB, DD, 5, bias_scale=0.3)
    ref = dss.forward(g.xy, g.n_int, g.src, g.dst, c, w, KB, DD, 0.2, hbar)
    n = g.xy.shape[0]
    rng = np.random.default_rng(0)
    perm_int = rng.permutation(g.n_int)
    perm = np.concatenate([perm_int, g.n_int + rng.permutation(n - g.n_int)])
    inv = np.argsort(perm)                       # new id of old node
    out = dss.forward(g.xy[perm], g.n_int, inv[g.src], inv[g.dst], c[perm_int], w, KB, DD, 0.2, hbar)
    assert np.allclose(out, ref[perm_int], rtol=1e-12, atol=1e-14)
    out = dss.forward(g.xy + np.array([3.5, -7.25]), g.n_int, g.src, g.dst, c, w, KB, DD, 0.2, hbar)
    assert np.allclose(out, ref, rtol=1e-11, atol=1e-13)


def test_reflection_swaps_the_two_message_directions():
    """On a graph without halo (all edges both ways), reflecting x -> -x turns d_jl into d_lj:
    the model with Phi_out and Phi_in exchanged (and Psi's two message inputs exchanged)
    gives the same output.  A sign error in either edge feature breaks this."""
    m = synth.square_mesh(7, seed=9)
    edges, _ = fem.mesh_edges(m.tri)
    src = np.concatenate([edges[:, 0], edges[:, 1]])
    dst = np.concatenate([edges[:, 1], edges[:, 0]])
    c = synth.residual_vector(m.n, 11)
    d = 5
    w = synth.dss_weights(3, d, 12, bias_scale=0.3).astype(np.float64)
    blocks = dss.unpack(w, 3, d)
    swapped = []
    for blk in blocks:
        for name, _shape in dss.block_shapes(d):
            if name.startswith("phi_out"):
                v = blk["phi_in" + name[7:]]
            elif name.startswith("phi_in"):
                v = blk["phi_out" + name[6:]]
            elif name == "psi.W1":
                v = blk[name].copy()
                v[:, d + 1:2 * d + 1], v[:, 2 * d + 1:] = blk[name][:, 2 * d + 1:], blk[name][:, d + 1:2 * d + 1]
            else:
                v = blk[name]
            swapped.append(np.ravel(v))
    w2 = np.concatenate(swapped)
    a = dss.forward(m.xy, m.n, src, dst, c, w, 3, d, 0.3, 0.1)
    b = dss.forward(-m.xy, m.n, src, dst, c, w2, 3, d, 0.3, 0.1)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-14)
    # and the unswapped model does see the reflection
    b0 = dss.forward(-m.xy, m.n, src, dst, c, w, 3, d, 0.3, 0.1)
    assert not np.allclose(a, b0, rtol=1e-6)
