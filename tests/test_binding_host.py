"""Argument checks of the Python binding (no GPU needed).  The C ABI takes
bare device pointers, so the binding refuses tensors of the wrong type or of
too few words (sign vectors, outputs, batch code outputs and batch jobs'
own sign vectors) before it hands them to the library; these checks run before
any library call, so CPU tensors and a triangulation object built without a
device reach every one of them."""
import pytest

torch = pytest.importorskip("torch")

import paper_2604_09221_gb300 as eng


def fake_tri(sign_words, code_words):
    t = object.__new__(eng.Triangulation)
    t._h = None
    t.d = 10
    t.sign_words, t.code_words = sign_words, code_words
    return t


def test_real_schemes_rejects_bad_tensors():
    t = fake_tri(2, 2)
    with pytest.raises(ValueError, match="multiple of sign_words"):
        t.real_schemes(torch.zeros(7, dtype=torch.int64))
    with pytest.raises(ValueError, match="10 words, 12 needed"):   # out one row short
        t.real_schemes(torch.zeros((6, 2), dtype=torch.int64), out=torch.zeros((5, 2), dtype=torch.int64))
    with pytest.raises(ValueError, match="64-bit integer"):
        t.real_schemes(torch.zeros((6, 2), dtype=torch.int64), out=torch.zeros((6, 2), dtype=torch.int32))
    with pytest.raises(ValueError, match="64-bit integer"):
        t.real_schemes(torch.zeros((6, 2), dtype=torch.int64), out=torch.zeros((6, 2), dtype=torch.float64))
    with pytest.raises(ValueError, match="contiguous"):
        t.real_schemes(torch.zeros((6, 2), dtype=torch.int64), out=torch.zeros((2, 6), dtype=torch.int64).t())
    with pytest.raises(ValueError, match="CUDA"):
        t.real_schemes(torch.zeros((6, 2), dtype=torch.int64))
    with pytest.raises(ValueError, match="CUDA"):
        t.real_schemes(torch.zeros((6, 2), dtype=torch.int64), out=torch.zeros((6, 2), dtype=torch.int64))


def test_splitmix_masks_rejects_a_short_output():
    # d = 10: |A| = 66 points, two words per sign vector
    with pytest.raises(ValueError, match="199 words, 200 needed"):
        eng.splitmix_masks(10, 0, 100, out=torch.zeros(199, dtype=torch.int64))
    with pytest.raises(ValueError, match="64-bit integer"):
        eng.splitmix_masks(7, 0, 100, out=torch.zeros(100, dtype=torch.int32))


def test_batch_rejects_mismatched_jobs_and_short_outputs():
    tris = [fake_tri(1, 1), fake_tri(3, 4)]
    with pytest.raises(ValueError, match="one entry per job"):
        eng.Batch(tris, [10], [0, 1])
    with pytest.raises(ValueError, match="one entry per job"):
        eng.Batch(tris, [10, 20], [0, 1], code_outputs=[None])
    with pytest.raises(ValueError, match="79 words, 80 needed"):   # 20 vectors x 4 code words
        eng.Batch(tris, [10, 20], [0, 1],
                  code_outputs=[None, torch.zeros(79, dtype=torch.int64)])


def test_batch_set_signs_rejects_bad_tensors():
    import numpy as np
    b = object.__new__(eng.Batch)
    b._h = None
    b.tris = [fake_tri(2, 2)]
    b.counts = np.array([10], dtype=np.uint64)
    with pytest.raises(ValueError, match="19 words, 20 needed"):   # 10 vectors x 2 sign words
        b.set_signs(0, torch.zeros(19, dtype=torch.int64))
    with pytest.raises(ValueError, match="64-bit integer"):
        b.set_signs(0, torch.zeros(20, dtype=torch.int32))
    with pytest.raises(ValueError, match="CUDA"):
        b.set_signs(0, torch.zeros(20, dtype=torch.int64))
