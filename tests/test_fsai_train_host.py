"""Host logic of the learned-FSAI driver: stored weights load from fp32 values or bf16
bit patterns into the parameter layout, the untrained network is Jacobi's, and the
gain summary's ratios are formed per matrix before the median."""
import numpy as np
import pytest

from paper_2608_09647_gb300 import fsai_train
from paper_2608_09647_gb300 import CG_MLP_PARAMS


def test_init_params_has_a_zero_output_layer():
    p = fsai_train.init_params(3)
    assert p.dtype == np.float32 and p.size == CG_MLP_PARAMS
    assert np.all(p[-65:] == 0)                  # w3 (64) and b3: the output o is 0, G = D^-1/2


def test_load_params_reads_fp32_and_bf16_bits(tmp_path):
    p = fsai_train.init_params(5)
    f32 = tmp_path / "p32.npy"
    np.save(f32, p)
    assert np.array_equal(fsai_train.load_params(str(f32)), p)
    bits = (p.view(np.uint32) >> 16).astype(np.uint16)   # truncation: exact for bf16-representable values
    p_bf = (bits.astype(np.uint32) << 16).view(np.float32)
    fb = tmp_path / "pbf.npy"
    np.save(fb, bits)
    assert np.array_equal(fsai_train.load_params(str(fb)), p_bf)
    bad = tmp_path / "bad.npy"
    np.save(bad, p[:10])
    with pytest.raises(ValueError):
        fsai_train.load_params(str(bad))


def test_committed_weights_load():
    import os
    w = os.path.join(os.path.dirname(fsai_train.__file__), "fsai_q1aniso_bf16.npy")
    p = fsai_train.load_params(w)
    assert p.size == CG_MLP_PARAMS and np.all(np.isfinite(p)) and np.any(p[-65:] != 0)


def test_summary_ratios_are_per_matrix():
    rows = []
    for k, (j64, ls, lset) in enumerate([(10.0, 4.0, 1.0), (20.0, 5.0, 1.0), (30.0, 9.0, 3.0)]):
        rows.append({"jacobi_iters": 100, "jacobi_s": 8.0, "jacobi64_s": j64, "classic_iters": 50, "classic_s": 5.0,
                     "learned_iters": 40 + k, "learned_s": ls, "learned_setup_s": lset})
    s = fsai_train.summarize(rows)
    assert s["learned_vs_jacobi64_time"]["median"] == pytest.approx(0.3)        # 0.4, 0.25, 0.3
    assert s["learned_setup_plus_solve_vs_jacobi64_time"]["median"] == pytest.approx(0.4)  # 0.5, 0.3, 0.4
    assert s["learned_vs_jacobi_iters"]["median"] == pytest.approx(0.41)
    assert s["learned_vs_classic_iters"]["q1"] <= s["learned_vs_classic_iters"]["median"] <= \
        s["learned_vs_classic_iters"]["q3"]
