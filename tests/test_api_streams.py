"""Host logic of the Python binding (no GPU): every call that takes a stream
runs with it as PyTorch's current stream, whether the stream is passed by
keyword or by position, and leaves the current stream alone without one."""
import contextlib

import pytest

from paper_2010_00465_gb300 import api


@pytest.fixture
def entered(monkeypatch):
    log = []

    @contextlib.contextmanager
    def fake_stream(s):
        log.append(("enter", s))
        try:
            yield
        finally:
            log.append(("exit", s))

    monkeypatch.setattr(api.torch.cuda, "stream", fake_stream)
    return log


def test_stream_by_keyword_and_position(entered):
    seen = []

    @api._on_stream
    def call(a, prec=None, stream=None):
        seen.append((a, prec, stream, list(entered)))
        return a

    marker = object()
    assert call(1, "fp64", stream=marker) == 1
    assert seen[-1][3] == [("enter", marker)]
    assert entered[-1] == ("exit", marker)
    entered.clear()
    assert call(2, "fp64", marker) == 2  # positional stream
    assert seen[-1][3] == [("enter", marker)]
    entered.clear()
    assert call(3) == 3  # no stream: no context
    assert entered == [] and seen[-1][2] is None


def test_exit_on_error(entered):
    @api._on_stream
    def call(stream=None):
        raise ValueError("bad argument")

    marker = object()
    with pytest.raises(ValueError):
        call(stream=marker)
    assert entered == [("enter", marker), ("exit", marker)]


def test_public_calls_are_wrapped():
    import inspect
    for name in ("norm1", "cossin", "cossin_cs", "matmul", "cossin_backward", "unitary", "unitary_backward",
                 "cossin_batched"):
        fn = getattr(api, name)
        assert "stream" in inspect.signature(fn).parameters, name
        assert hasattr(fn, "__wrapped__"), name  # functools.wraps of _on_stream
    assert hasattr(api.BatchedPlan.__init__, "__wrapped__")
