"""The bench's fixed settings against the binding's signatures (no GPU).

The bench passes its training, form and estimator settings as keyword
arguments; a name that drifts from the binding would only fail on the GPU
box.  These checks catch that here.
"""
import importlib
import inspect
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    return importlib.import_module("bench")


def test_training_settings_are_surrogate_train_arguments(bench):
    import paper_1910_04727_gb300 as fm
    params = inspect.signature(fm.Context.surrogate_train).parameters
    for name in ("SURROGATE_TRAIN", "C5_TRAIN"):
        for key in getattr(bench, name):
            assert key in params, (name, key)
    # the training pairs are solved to a looser tolerance than the estimator's
    assert 0 < bench.SURROGATE_TRAIN["target_tol"] < 1e-4
    assert bench.SURROGATE_TRAIN["n_train"] % bench.SURROGATE_TRAIN["batch"] == 0


def test_forms_are_context_settings(bench):
    import paper_1910_04727_gb300 as fm
    params = inspect.signature(fm.Context.__init__).parameters
    for form, f in bench.FORMS.items():
        assert f["precision"] in (0, 1), form
        assert "precision" in params and "converged" in params
        # the mixed form always refines to a tolerance
        assert f["precision"] == 0 or f["converged"], form


def test_command_line_flags_parse(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "2", "--warmup", "3", "--train-tol", "1e-6",
                                      "--surrogate-cost", "0.01", "--train-n", "4096"])
    args = bench.parse()
    assert args.steps == 2 and args.warmup == 3
    assert args.train_tol == 1e-6 and args.surrogate_cost == 0.01 and args.train_n == 4096
