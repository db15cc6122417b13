"""Host logic of the Python binding (no GPU): a Network keeps its marshalled C form
between calls while it holds the same tensor objects over the same storage, the same
edges and the same open modes, and rebuilds it when any of them changes; the cached
form stays out of pickles and copies."""
import copy
import pickle

import pytest

from paper_2603_07387_gb300 import tnsk

torch = pytest.importorskip("torch")


def _net():
    A, B, C = (torch.ones(4, 4) for _ in range(3))
    return tnsk.Network([A, B, C], [(1, 2), (3, 4), (5, 0)], [])


def test_marshalled_form_is_reused_while_unchanged():
    n = _net()
    h = tnsk._holder(n)
    assert tnsk._holder(n) is h
    assert h.c.p == 3 and h.c.t == 3 and h.c.n_open == 0
    assert [h.edges[i] for i in range(6)] == [1, 2, 3, 4, 5, 0]
    assert h.tens[0].data == n.tensors[0].data_ptr()


@pytest.mark.parametrize("change", ["tensor", "storage", "edges", "open"])
def test_marshalled_form_is_rebuilt_on_change(change):
    n = _net()
    h = tnsk._holder(n)
    if change == "tensor":
        n.tensors[1] = torch.zeros(4, 4)
    elif change == "storage":
        n.tensors[2].set_(torch.zeros(4, 4))
    elif change == "edges":
        n.edges = [(1, 2), (3, 4)]
        n.open = [5, 0]
    else:
        n.edges = [(1, 2), (3, 4)]
        n.open = [0, 5]
    h2 = tnsk._holder(n)
    assert h2 is not h
    assert [h2.tens[k].data for k in range(3)] == [t.data_ptr() for t in n.tensors]
    assert h2.c.t == len(n.edges) and h2.c.n_open == len(n.open)
    if change == "open":  # the same edges as the "edges" case, another output order
        assert [h2.open[i] for i in range(2)] == [0, 5]


def test_marshalled_form_stays_out_of_pickles_and_copies():
    n = _net()
    tnsk._holder(n)
    for m in (pickle.loads(pickle.dumps(n)), copy.deepcopy(n)):
        assert "_holder" not in m.__dict__
        assert m.edges == n.edges
        h = tnsk._holder(m)
        assert h.c.p == 3


def test_schedule_json_table_round_trip(tmp_path):
    """A scatter schedule (what tnsk_autotune finds) saved as a JSON table and loaded for
    later plans is the same schedule; malformed tables are refused."""
    s = tnsk.Schedule()
    s.rep_cap[:] = [(3 * i) % 33 for i in range(tnsk.SCATTER_LISTS)]
    s.chunk_scale[:] = [1 + i % 4 for i in range(tnsk.SCATTER_LISTS)]
    path = str(tmp_path / "schedule.json")
    s.save(path)
    t = tnsk.Schedule.load(path)
    assert t.as_dict() == s.as_dict()
    with pytest.raises(ValueError):
        tnsk.Schedule.from_dict({"rep_cap": [1, 2], "chunk_scale": [1, 2]})
    with pytest.raises(ValueError):
        tnsk.Schedule.from_dict({"rep_cap": [-1] * tnsk.SCATTER_LISTS, "chunk_scale": [1] * tnsk.SCATTER_LISTS})
