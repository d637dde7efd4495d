"""The seeded synthetic parameter sets: the library's generator (C++,
sd_load_energy with no file) and the test suite's (Python, inputs.py) draw the
same SplitMix64 numbers in the same recipe, so they must write byte-identical
parameter files.  The C++ side is compiled here with a small shim (host code
only, no GPU).  The GPU test closes the loop: a design with the seeded set
loaded inside the library equals the oracle's design on the Python-written
file, bit for bit.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2609_32308_b300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2609_32308_b300", "csrc", "sd_synth.cpp")

SHIM = r"""
#include <cstdint>
#include <cstring>
#include <string>
std::string sd_internal_synthetic_text(uint64_t seed);
extern "C" int synth_text(uint64_t seed, char *buf, int cap) {
  const std::string s = sd_internal_synthetic_text(seed);
  if ((int)s.size() + 1 > cap) return -1;
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return (int)s.size();
}
"""


@pytest.fixture(scope="module")
def csynth(tmp_path_factory):
    d = tmp_path_factory.mktemp("synth")
    shim = d / "shim.cpp"
    shim.write_text(SHIM)
    so = d / "libsynth.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", str(so), SRC,
                           str(shim)])
    lib = ctypes.CDLL(str(so))
    lib.synth_text.argtypes = [ctypes.c_uint64, ctypes.c_char_p, ctypes.c_int]
    buf = ctypes.create_string_buffer(1 << 20)

    def text(seed):
        n = lib.synth_text(seed, buf, len(buf))
        assert n > 0
        return buf.value.decode()
    return text


@pytest.mark.parametrize("seed", [0, 1, 7, 123456789, 2**63 + 5])
def test_c_and_python_generators_write_the_same_file(csynth, seed):
    assert csynth(seed) == inputs.energy_text(inputs.synthetic_energy_params(seed))


def test_generated_tables_have_the_model_symmetries(csynth):
    from oracle.params import read_params
    import tempfile
    with tempfile.NamedTemporaryFile("w", suffix=".par", delete=False) as f:
        f.write(csynth(11))
    P = read_params(f.name)
    os.unlink(f.name)
    st = np.asarray(P["stack"])
    assert np.array_equal(st, st.T)
    i11 = np.asarray(P["int11"])
    assert np.array_equal(i11, i11.transpose(1, 0, 3, 2))
    i22 = np.asarray(P["int22"])
    assert np.array_equal(i22, i22.transpose(1, 0, 4, 5, 2, 3))
    assert all(np.all(np.diff(np.asarray(P[n])[k:]) >= 0)
               for n, k in (("hairpin", 3), ("bulge", 1), ("interior", 2)))
    assert len(P["tetraloop"]) == 30 and len(P["triloop"]) == 20 and len(P["hexaloop"]) == 4


@pytest.mark.gpu
def test_seeded_energy_in_the_library_matches_the_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2609_32308_b300 as sd
    seed = 424
    E = sd.sd_load_energy(None, seed)
    saved = tmp_path / "saved.par"
    E.save(str(saved))
    par = inputs.synthetic_energy_file(seed, str(tmp_path))
    assert saved.read_text() == open(par).read()
    # the saved file loads back to the same designs
    E2 = sd.sd_load_energy(str(saved))
    for A, s, lam in ((40, 91, 4.0), (30, 92, 0.0)):
        prot = inputs.random_protein(A, s)
        w = inputs.random_codon_weights(s)
        r = sd.sd_design(E, prot, w, lam)
        o = oracle.run(par, prot, w, lam)
        assert (r["mrna"], r["structure"], r["energy"], r["objective_fx"]) == \
            (o.mrna, o.structure, o.energy, o.obj_fx)
        assert sd.sd_design(E2, prot, w, lam)["mrna"] == r["mrna"]
