"""The binding's size checks, without a GPU.  The library receives bare
pointers, so every row count, column count and caller-supplied output buffer
is checked in Python before the call; a mis-shaped tensor must raise there
rather than be read or written past its end on the device.

CPU tensors stand in for device tensors (``Tensor.is_cuda`` is patched for
these tests only) and the handles carry NULL pointers: every case must be
refused by the binding itself (ValueError/TypeError).  Were a check missing,
the call would reach the library with a NULL handle and fail differently."""

import pytest
import torch


@pytest.fixture(scope="module")
def fgk():
    from paper_2508_01864_gb300 import build, fgk

    build.build()
    fgk.load()
    return fgk


@pytest.fixture(autouse=True)
def cpu_as_device(monkeypatch):
    monkeypatch.setattr(torch.Tensor, "is_cuda", property(lambda self: True), raising=False)


N, D = 10, 2


def f64(*shape):
    return torch.zeros(*shape, dtype=torch.float64)


def f32(*shape):
    return torch.zeros(*shape, dtype=torch.float32)


@pytest.fixture
def h(fgk):
    return fgk.Handle(0, N, D, 3, fgk.FGK_PRODUCT)


@pytest.fixture
def pc(fgk, h):
    return fgk.Precond(0, h, 0.01, rank=4)


def test_products_check_rows_and_the_output_buffer(fgk, h):
    for call in (lambda V, **k: fgk.fgk_matvec(h, V, "f64", **k),
                 lambda V, **k: fgk.fgk_matvec_dlogell(h, V, 0, "f64", **k),
                 lambda V, **k: fgk.fgk_matvec_q(h, V, "f64", **k)):
        with pytest.raises(ValueError, match="rows"):
            call(f64(N + 1, 2))
        with pytest.raises(ValueError, match="shape"):
            call(f64(N, 2), out=f64(N, 1))
        with pytest.raises(ValueError, match="shape"):
            call(f64(N, 2), out=f64(N * 2))  # same bytes, wrong shape
        with pytest.raises(TypeError):
            call(f64(N, 2), out=f32(N, 2))
        with pytest.raises(TypeError):
            call(f64(N, 2), out=f64(2, N).t())  # not contiguous


def test_no_alloc_product_needs_a_matching_buffer(fgk, h):
    with pytest.raises(TypeError, match="required"):
        fgk.fgk_matvec_q_noalloc(h, f32(N, 1), None)
    with pytest.raises(ValueError, match="shape"):
        fgk.fgk_matvec_q_noalloc(h, f32(N, 3), f32(N, 1))
    with pytest.raises(ValueError, match="rows"):
        fgk.fgk_matvec_q_noalloc(h, f32(N - 1, 1), f32(N - 1, 1))


def test_out_for_accepts_a_vector_for_one_column_and_writes_in_place(fgk):
    like = f64(N, 1)
    out = f64(N)
    view = fgk._out_for(out, like)
    assert view.shape == (N, 1) and view.data_ptr() == out.data_ptr()
    view.fill_(2.0)
    assert float(out.sum()) == 2.0 * N
    with pytest.raises(ValueError):
        fgk._out_for(f64(N), f64(N, 2))


def test_solve_checks_rows_of_y_and_h(fgk, h):
    with pytest.raises(ValueError, match="y has"):
        fgk.fgk_cg_solve(h, f64(N + 3), 0.01)
    with pytest.raises(ValueError, match="H has"):
        fgk.fgk_cg_solve(h, f64(N), 0.01, H=f64(N - 1, 3))


def test_preconditioner_calls_check_sizes(fgk, pc):
    with pytest.raises(ValueError, match="R has"):
        fgk.fgk_precond_apply(pc, f64(N + 1, 2))
    with pytest.raises(ValueError, match="shape"):
        fgk.fgk_precond_apply(pc, f64(N, 2), out=f64(N, 3))
    with pytest.raises(ValueError, match="E_n has"):
        fgk.fgk_precond_sample(pc, f64(4, 3), f64(N + 1, 3))
    with pytest.raises(ValueError, match="E_r has 5 rows"):
        fgk.fgk_precond_sample(pc, f64(5, 3), f64(N, 3))
    with pytest.raises(ValueError, match="columns"):
        fgk.fgk_precond_sample(pc, f64(4, 2), f64(N, 3))


def test_likelihood_calls_check_sizes(fgk, h):
    with pytest.raises(ValueError, match="B has"):
        fgk.fgk_slq_logdet(h, f64(N - 2, 4), 0.01, 20)
    with pytest.raises(ValueError, match="y has"):
        fgk.fgk_loglik_grad(h, f64(N + 1), f64(N, 4), 0.01)
    with pytest.raises(ValueError, match="one column"):
        fgk.fgk_loglik_grad(h, f64(N, 2), f64(N, 4), 0.01)
    with pytest.raises(ValueError, match="B has"):
        fgk.fgk_loglik_grad(h, f64(N), f64(N + 1, 4), 0.01)


def test_predict_checks_alpha_covariates_and_beta(fgk, h):
    Z = f64(7, D)
    with pytest.raises(ValueError, match="alpha has"):
        fgk.fgk_predict(h, f64(N + 1), Z)
    with pytest.raises(ValueError, match="HZ has"):
        fgk.fgk_predict(h, f64(N), Z, HZ=f64(6, 3), beta=f64(3, 1))
    with pytest.raises(ValueError, match="beta has shape"):
        fgk.fgk_predict(h, f64(N), Z, L=-1, beta=f64(2, 1))  # the default [1, z] has 1 + d rows
    with pytest.raises(ValueError, match="beta has shape"):
        fgk.fgk_predict(h, f64(N, 2), Z, HZ=f64(7, 3), beta=f64(3, 1))  # one column per right-hand side


def test_batch_calls_check_every_problem(fgk):
    hs = [fgk.Handle(0, 10, 1, 3, 1), fgk.Handle(0, 15, 2, 3, 1)]
    b = fgk.Batch(0, hs, 2, [0, 10, 25])
    with pytest.raises(TypeError):
        fgk.fgk_batch_matvec_q(b, f32(24, 2))
    with pytest.raises(ValueError, match="shape"):
        fgk.fgk_batch_matvec_q(b, f32(25, 2), out=f32(25, 1))
    with pytest.raises(ValueError, match="2 problems"):
        fgk.fgk_batch_cg_solve(b, [f64(10, 2)], [0.01, 0.01])
    with pytest.raises(ValueError, match="2 problems"):
        fgk.fgk_batch_cg_solve(b, [f64(10, 2), f64(15, 2)], [0.01])
    with pytest.raises(ValueError, match="y has 14 rows"):
        fgk.fgk_batch_cg_solve(b, [f64(10, 2), f64(14, 2)], [0.01, 0.01])
    with pytest.raises(ValueError, match="columns"):
        fgk.fgk_batch_cg_solve(b, [f64(10, 2), f64(15, 1)], [0.01, 0.01])
