"""Host-side parts of the server (no GPU): the start-up warm-up of the reference elements."""
import pytest

from paper_2506_17406_gb300 import riesz as rz
from paper_2506_17406_gb300 import serve


def test_server_warm_builds_every_pair():
    """warm() creates one host-only handle per (space, degree) with the server's options (the paper's
    decomposition per space, so the Hiptmair-Toselli potential spaces are built too) from several
    threads and reports each handle's host time; every pair asked for is there."""
    srv = serve.Server(recommended=True)
    spaces, degrees = ("CG", "RT", "N2curl"), (1, 2)
    out = srv.warm(spaces, degrees, threads=3)
    assert set(out) == {(s, p) for s in spaces for p in degrees}
    assert all(ms >= 0.0 for ms in out.values())


def test_server_warm_rejects_an_unknown_space():
    with pytest.raises(Exception):
        serve.Server(recommended=True).warm(("H3",), (1,))
