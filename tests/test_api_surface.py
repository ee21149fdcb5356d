"""The Python names the README's examples use exist in the binding, with the
options they pass (no GPU needed: the library is only loaded, not run)."""
import paper_1210_2536_gb300 as smat


def test_documented_python_names_exist():
    for name in ("SpMatrix", "Batch", "Segments", "cg_mixed", "plan_cache_save", "plan_cache_load",
                 "plan_cache_clear", "plan_cache_size", "smat_load_model", "smat_measure_gather_rate",
                 "MODEL_PATH", "SMAT_BATCH_AUTO", "SMAT_BATCH_GRAPH", "SMAT_BATCH_PER_MATRIX"):
        assert hasattr(smat, name), name
    for name in ("tune", "spmv", "plan", "plan_key", "features", "timings", "launches", "export_parts", "close"):
        assert hasattr(smat.SpMatrix, name), name


def test_documented_options_are_struct_fields():
    tune = {n for n, _ in smat.smat_tune_opts_t._fields_}
    assert {"plan_cache", "trial_race", "trial_extended", "sell_sigma", "allowed", "trial_reps"} <= tune
    batch = {n for n, _ in smat.smat_batch_opts_t._fields_}
    assert {"tile_scale", "ctas_per_sm", "trial_reps", "mode"} <= batch
    cg = {n for n, _ in smat.smat_cg_opts_t._fields_}
    assert "rtol" in cg
