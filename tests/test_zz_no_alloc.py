"""The allocation-free entry point against the ordinary one (marked gpu).

sd_design_noalloc serves callers that may not allocate device memory when
they ask for a design: it runs the same kernels inside a scratch array the
library holds for the life of the process.  Two calls in a row must each give
exactly what sd_design gives (the second call reuses the scratch the first
left behind), and a design too large for the scratch must be refused.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2609_32308_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2609_32308_b300 as sd
    sd.lib()
    return sd


def test_noalloc_matches_sd_design_on_two_calls_in_a_row(sd, par1):
    E = sd.sd_load_energy(par1)
    cases = [(inputs.random_protein(60, 71), inputs.random_codon_weights(71), 4.0),
             (inputs.random_protein(23, 72), inputs.random_codon_weights(72), 0.0)]
    for prot, w, lam in cases:
        got = sd.sd_design_noalloc(E, prot, w, lam)
        ref = sd.sd_design(E, prot, w, lam)
        assert got["status"] == ref["status"] == 0
        for key in ("mrna", "structure", "energy", "objective_fx", "codon_cost", "objective",
                    "Z", "finite_direct", "retained_cells", "states", "edges", "n"):
            assert got[key] == ref[key], key
        assert abs(got["objective"] - ref["objective"]) <= 1e-9


def test_noalloc_refuses_designs_larger_than_its_scratch(sd, par1):
    E = sd.sd_load_energy(par1)
    prot = inputs.random_protein(300, 73)
    with pytest.raises(sd.SdError) as ei:
        sd.sd_design_noalloc(E, prot, inputs.random_codon_weights(73), 4.0)
    assert ei.value.code == sd.SD_ESIZE
    # and it still works afterwards
    small = inputs.random_protein(12, 74)
    w = inputs.random_codon_weights(74)
    assert sd.sd_design_noalloc(E, small, w, 1.0)["mrna"] == sd.sd_design(E, small, w, 1.0)["mrna"]


def test_noalloc_edge_sizes(sd, par1):
    """The empty protein, one codon, a stop codon alone and two codons give
    exactly what sd_design gives."""
    E = sd.sd_load_energy(par1)
    w = inputs.random_codon_weights(75)
    for prot in ("", "M", "*", "MW"):
        got = sd.sd_design_noalloc(E, prot, w, 4.0)
        ref = sd.sd_design(E, prot, w, 4.0)
        for key in ("status", "mrna", "structure", "energy", "objective_fx", "n"):
            assert got[key] == ref[key], (prot, key)
