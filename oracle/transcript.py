"""Record of openings (communication rounds) performed by the protocol.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Table 3 of the paper counts round complexity: the number of sequential
round-trips of communication.  Every reveal of a masked value (epsilon/delta of
a Beaver product, the masks of a binary AND, z of Alg. 2) is one opening.
Openings that the protocol performs in parallel belong to the same round; the
caller states the round boundary with ``next_round``.
"""


class Transcript:
    def __init__(self):
        self.rounds = 0
        self.openings = 0
        self.bytes_per_party = 0
        self._open_in_round = False

    def open(self, nbytes_per_party):
        """Record one opening of nbytes per party in the current round."""
        if not self._open_in_round:
            self.rounds += 1
            self._open_in_round = True
        self.openings += 1
        self.bytes_per_party += int(nbytes_per_party)

    def next_round(self):
        self._open_in_round = False


def _maybe(tr):
    return tr if tr is not None else Transcript()
