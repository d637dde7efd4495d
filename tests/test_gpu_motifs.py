"""Forbidden-motif product automata on the GPU against the oracle (marked gpu).

The codon DFA intersected with the motifs' Aho-Corasick automaton keeps the
layered path model (Sec. 3), so every table of the exact DP on the product
must equal the dense oracle's on its own, independently built product, cell by
cell (narrow products run on the plain kernels, wider ones on the wide
instance with forward-packed tables), and the designs must contain no motif.
"""
import numpy as np
import pytest

import oracle
from oracle import evaluate
from oracle.params import read_params
from paper_2609_32308_b300 import inputs

from test_gpu_parity import compare_design, compare_tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2609_32308_b300 as sd
    sd.lib()
    return sd


@pytest.fixture(scope="module")
def E1(sd, par1):
    return sd.sd_load_energy(par1)


CASES = [(40, 61, 4.0, ["AAUAAA"]),
         (40, 62, 0.0, ["GGUAAG", "AAUAAA", "UUUUU"]),
         (60, 63, 4.0, ["CUG", "GCU", "AGC", "CGC"]),
         (50, 64, 4.0, ["GAAUUC", "GGAUCC", "AAGCUU", "CUCGAG", "CCCGGG", "GGCC"]),
         (30, 66, 1.5, ["CCCCCCCC"])]


@pytest.mark.parametrize("A,seed,lam,motifs", CASES)
def test_motif_tables_and_design_match_the_oracle(sd, E1, par1, A, seed, lam, motifs):
    prot = inputs.random_protein(A, seed)
    w = inputs.random_codon_weights(seed)
    o = oracle.run_motifs(par1, prot, w, lam, motifs)
    assert o is not None and o.status == 0
    plan = sd.Plan(E1, [prot], w, [lam], motifs=motifs)
    e = plan.edges(0)
    assert e["from"].tolist() == o.edge_from.tolist() and e["to"].tolist() == o.edge_to.tolist()
    assert e["label"].tolist() == o.edge_label.tolist()
    assert e["cost"].tolist() == o.edge_cost.tolist()
    plan.run()
    r = plan.results()[0]
    compare_tables(plan, 0, o)
    compare_design(r, o, lam)
    assert not any(m in r["mrna"] for m in motifs)
    assert evaluate.energy(read_params(par1), r["mrna"], r["structure"]) == r["energy"]
    plain = sd.sd_design(E1, prot, w, lam)
    assert r["objective_fx"] >= plain["objective_fx"]
    plan.free()


def test_motif_batch_under_graph_replay(sd, E1, par1):
    motifs = ["GAAUUC", "GGAUCC", "AAUAAA"]
    batch = inputs.protein_batch([30, 12, 45, 20, 3], seed=321)
    plan = sd.Plan(E1, [b[0] for b in batch], np.stack([b[1] for b in batch]),
                   [b[2] for b in batch], motifs=motifs)
    plan.set_graph(True)
    for _ in range(2):
        plan.run()
        for (p, w, lam), r in zip(batch, plan.results()):
            compare_design(r, oracle.run_motifs(par1, p, w, lam, motifs), lam)
    plan.free()


def test_motif_edge_cases(sd, E1, par1):
    w = inputs.random_codon_weights(44)
    prot = inputs.random_protein(30, 44)
    # no motif: the plain design
    a = sd.sd_design_motifs(E1, prot, w, 4.0, [])
    b = sd.sd_design(E1, prot, w, 4.0)
    assert (a["mrna"], a["objective_fx"]) == (b["mrna"], b["objective_fx"])
    # an unavoidable motif: empty design language
    with pytest.raises(sd.SdError) as ei:
        sd.sd_design_motifs(E1, "MW", w, 1.0, ["GU"])
    assert ei.value.code == sd.SD_EINFEASIBLE
    plan = sd.Plan(E1, ["MW", "MK"], w, [1.0, 1.0], motifs=["GU"])
    assert plan.item_status.tolist() == [sd.SD_EINFEASIBLE, 0]
    plan.run()
    res = plan.results()
    assert res[0]["status"] == sd.SD_EINFEASIBLE
    compare_design(res[1], oracle.run_motifs(par1, "MK", w, 1.0, ["GU"]), 1.0)
    # malformed motifs
    for bad in (["ACGT"], [""], ["A" * 33]):
        with pytest.raises(sd.SdError) as ei:
            sd.sd_design_motifs(E1, prot, w, 1.0, bad)
        assert ei.value.code == sd.SD_EINVAL
