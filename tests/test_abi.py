"""The C-ABI library builds, loads and exports every symbol of include/sf_eprl.h; host-only
helpers (ranges, shell counts, argument validation) agree with the oracle. No device work."""
import os
import re

import pytest

import paper_2107_13952_gb300 as sf
from oracle import vertex as ov
from paper_2107_13952_gb300 import inputs

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sf_eprl.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sf_[a-z0-9_]+)\s*\(", src)))


def test_header_matches_binding_exports():
    assert declared_functions() == sorted(sf.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = sf.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert b"sm_103a" in lib.sf_version()


@pytest.mark.parametrize("seed", range(5))
def test_intertwiner_ranges_match_oracle(seed):
    for v in inputs.random_batch(n=20, seed=seed):
        lo, dim = sf.intertwiner_ranges(v["two_j"], v["gamma"], v["dl"])
        ref = ov.intertwiner_ranges(v["two_j"])
        assert dim == [len(r) for r in ref]
        assert lo == [r[0] for r in ref]
        assert sf.num_shells(v["two_j"], v["gamma"], v["dl"]) == ov.n_shells(v["dl"])


def test_argument_validation():
    with pytest.raises(sf.SfError) as e:
        sf.intertwiner_ranges((1,) * 9 + (2,))
    assert e.value.code in (sf.SF_ERR_EMPTY, sf.SF_ERR_ARG)
    with pytest.raises(sf.SfError) as e:
        sf.num_shells((2,) * 10, 1.2, -1)
    assert e.value.code == sf.SF_ERR_ARG
    with pytest.raises(sf.SfError) as e:
        sf.num_shells((2,) * 10, -1.0, 1)
    assert e.value.code == sf.SF_ERR_ARG
    with pytest.raises(sf.SfError) as e:
        sf.num_shells((2,) * 10, 1.2, 1000)
    assert e.value.code == sf.SF_ERR_LIMIT


def test_precision_values_match_header():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    vals = dict((k, int(v)) for k, v in re.findall(r"\b(SF_FP64|SF_MIXED_FF|SF_MIXED_PX|SF_MIXED_TC|SF_MIXED)\s*=\s*(\d+)", src))
    assert vals == {"SF_FP64": sf.SF_FP64, "SF_MIXED": sf.SF_MIXED, "SF_MIXED_FF": sf.SF_MIXED_FF,
                    "SF_MIXED_TC": sf.SF_MIXED_TC, "SF_MIXED_PX": sf.SF_MIXED_PX}
