"""Host logic of the EMD-kNN driver: neighbour order and voting, and the
whole classifier on oracle distances (CPU)."""
import numpy as np

import oracle
from paper_2401_07378_gb300 import knn, workloads as wl


def test_nearest_orders_by_distance_then_index():
    d = np.array([3.0, 1.0, 2.0, 1.0, 0.5])
    assert knn.nearest(d, 4).tolist() == [4, 1, 3, 2]


def test_vote_majority_and_ties():
    labels = np.array([0, 1, 1, 2, 0])
    assert knn.vote(np.array([1.0, 2.0, 3.0, 9.0, 9.0]), labels, 3) == 1      # 1 twice
    # 0 and 1 once each among k = 2: the smaller summed distance wins
    assert knn.vote(np.array([2.0, 1.0, 5.0, 9.0, 9.0]), labels, 2) == 1
    # equal sums: the smaller label
    assert knn.vote(np.array([1.0, 1.0, 5.0, 9.0, 9.0]), labels, 2) == 0


def test_classifier_on_oracle_distances():
    docs = wl.labelled_documents(classes=3, docs_per_class=8, queries_per_class=2, seed=1, d=16)
    correct = 0
    for (y, b), lab in zip(docs.queries, docs.query_labels):
        dist = np.array([oracle.solve(docs.x[docs.x_off[p]:docs.x_off[p + 1]], docs.a[docs.x_off[p]:docs.x_off[p + 1]],
                                      y, b, "l2").cost for p in range(len(docs.labels))])
        correct += knn.vote(dist, docs.labels, 3) == lab
    assert correct == len(docs.query_labels)
