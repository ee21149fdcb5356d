"""The library's format selection against the oracle's, on the same seeded
matrices in each storage type: the admissibility filter (Sec. 2.3) as a mask
over the eight classes, the paper-rules pick (Sec. 4, in the order of Sec. 6;
``tune("rules")``) and the learned selector's pick and confidence without
trials (``tune("learned")`` with a confidence threshold of 0)."""
import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from helpers import csr_from_degrees, stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
VALUE_BYTES = {"f64": 8, "f32": 4, "bf16": 2}
LIB_ID = {"csr_scalar": smat.SMAT_V_CSR_SCALAR, "csr_vec4": smat.SMAT_V_CSR_VEC4, "csr_vec8": smat.SMAT_V_CSR_VEC8,
          "csr_vec32": smat.SMAT_V_CSR_VEC32, "csr_merge": smat.SMAT_V_CSR_MERGE, "ell": smat.SMAT_V_ELL,
          "dia": smat.SMAT_V_DIA, "coo": smat.SMAT_V_COO}


def _est_nnz(kind, p):
    if kind == synth.STENCIL2D5:
        return 5 * p[0] * p[1]
    if kind == synth.STENCIL3D7:
        return 7 * p[0] ** 3
    if kind == synth.STENCIL3D27:
        return 27 * p[0] ** 3
    if kind == synth.UNIFORM:
        return p[0] * p[1]
    if kind == synth.POWERLAW:
        return p[0] * synth.zipf_mean(p[1], int(p[2]))
    if kind == synth.BLOCKDIAG:
        return p[0] * p[1]
    return p[0] ** 3 * (2 * p[1] + 1) ** 3


def _matrices():
    mats = [synth.stencil2d5(64), synth.stencil3d7(12), synth.stencil3d27(16), synth.blockdiag(4096, 8, 0),
            synth.powerlaw(20000, 1.8, 1000, 3), synth.uniform_random(20000, 16.0, 1), synth.box3d(12, 3),
            csr_from_degrees([3] * 5000, 5000, 1), csr_from_degrees([12] * 3000, 3000, 2),
            csr_from_degrees([(2, 6)[i % 2] for i in range(4000)], 4000, 3),
            csr_from_degrees([(30, 34)[i % 2] for i in range(4000)], 4000, 3),
            csr_from_degrees([50 if i % 10 == 0 else 5 for i in range(2000)], 2000, 5)]
    picked = 0
    for mid in range(synth.DATASET_SIZE):
        kind, params, seed = synth.dataset_spec(mid)
        if _est_nnz(kind, params) <= 1.5e6:
            mats.append(synth.dataset_matrix(mid))
            picked += 1
        if picked == 40:
            break
    return mats


@pytest.fixture(scope="module")
def matrices():
    return [(A, oracle.features(A.m, A.n, A.rowptr, A.colidx)) for A in _matrices()]


def _oracle_mask(A, f, dtype):
    return oracle.admissible(A.m, A.nnz, f["max_rd"], f["ndiags"], VALUE_BYTES[dtype])


def _handle(A, dtype):
    vals, _ = stored_values(A, dtype)
    if dtype == "bf16":
        vals = vals.view(np.int16)
    return smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                         torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dtype)


def _lib_mask(oracle_mask):
    return sum(1 << LIB_ID[c] for i, c in enumerate(oracle.CLASSES) if (oracle_mask >> i) & 1)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_admissible_and_rules_pick_match_the_oracle(matrices, dtype):
    seen = set()
    for A, f in matrices:
        want = _oracle_mask(A, f, dtype)
        want_pick = LIB_ID[oracle.CLASSES[oracle.rules_select(f, want)]]
        M = _handle(A, dtype)
        assert M.features()["admissible"] & 0xFF == _lib_mask(want), (A.name, dtype)
        M.tune("rules", plan_cache=0)
        assert M.plan()["variant"] == want_pick, (A.name, dtype, M.plan()["name"])
        seen.add(want_pick)
        M.close()
    # the set reaches every rule: DIA, ELL, COO and CSR-vector
    assert {smat.SMAT_V_DIA, smat.SMAT_V_ELL, smat.SMAT_V_COO} <= seen
    assert seen & {smat.SMAT_V_CSR_VEC4, smat.SMAT_V_CSR_VEC8, smat.SMAT_V_CSR_VEC32}


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_learned_pick_matches_the_oracle(matrices, dtype):
    # the network runs in FP32 on the GPU and in FP64 in the oracle: where
    # the oracle's top probabilities lie within 1e-3 of each other, any of
    # them is the same decision
    assert smat.smat_load_model(smat.MODEL_PATH) == smat.SMAT_OK
    params, mean, std = smat.read_model(smat.MODEL_PATH)
    cls_of = {v: c for c, v in LIB_ID.items()}
    for A, f in matrices:
        want = _oracle_mask(A, f, dtype)
        best, p = oracle.learned_select(f, want, params, mean, std)
        M = _handle(A, dtype)
        M.tune("learned", conf_threshold=0.0, trial_extended=0, plan_cache=0)
        plan = M.plan()
        assert plan["trialled"] == 0, (A.name, dtype)
        c = oracle.CLASSES.index(cls_of[plan["variant"]])
        near = [k for k in range(len(oracle.CLASSES)) if p[k] >= p[best] - 1e-3]
        assert c in near, (A.name, dtype, plan["name"], oracle.CLASSES[best], p)
        assert abs(plan["confidence"] - p[c]) < 1e-3, (A.name, dtype, plan["confidence"], p[c])
        M.close()
